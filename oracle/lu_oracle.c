/*
 * CPU oracle for LU factorization with partial pivoting (PA = LU) and the
 * triangular solves that use it.  TEST INFRASTRUCTURE ONLY: it is called by the
 * tests, by the smoke check and by the benchmark's CPU-baseline leg, never by the
 * library.  It shares no code with the CUDA path.
 *
 * Plain, slow and deliberately unoptimised: IEEE double throughout, compiled
 * with -ffp-contract=off so every "a - l*u" is two roundings.
 *
 * Storage: column-major, element (i, j) at A[i + j*lda]; ipiv is 1-based with
 * LAPACK's sequential-interchange meaning (row j was interchanged with row
 * ipiv[j]-1 at step j).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(A, lda, i, j) (A)[(size_t)(i) + (size_t)(j) * (size_t)(lda)]

/* ------------------------------------------------------------------------ */
/* Unblocked right-looking LU with partial pivoting.
 *
 * Section 3.1, Figure 1 (left), LU_unb: for each column j,
 *   rl1: a21 := a21 / alpha11
 *   rl2: A22 := A22 - a21 * a12^T
 * with the standard partial pivoting that section 3.1 says every
 * implementation integrates: before rl1, the entry of largest magnitude in
 * column j (rows j..m-1) is brought to the diagonal by interchanging two full
 * rows.  Ties go to the smallest row index (the comparison is strict).  A zero
 * pivot records info = j+1 (first one only) and the column is left as is,
 * as LAPACK's getf2 does; the update with an all-zero a21 is a no-op.
 *
 * The rank-1 update is split over `nthreads` threads by columns of A22; each
 * element still sees exactly the same operations in the same order, so the
 * result does not depend on the thread count.
 * ------------------------------------------------------------------------ */

typedef struct {
    int m, n, lda;
    double *A;
    int nthreads;
    int tid;
    pthread_barrier_t *bar;
    volatile int *jstep;      /* current column, written by thread 0 */
    volatile int *skip;       /* 1 when the current pivot is zero */
} upd_arg;

static void rank1_cols(double *A, int lda, int m, int j, int c0, int c1)
{
    for (int c = c0; c < c1; ++c) {
        const double u = AT(A, lda, j, c);            /* a12 entry */
        for (int i = j + 1; i < m; ++i)
            AT(A, lda, i, c) = AT(A, lda, i, c) - AT(A, lda, i, j) * u;   /* rl2 */
    }
}

static void *upd_worker(void *p)
{
    upd_arg *a = (upd_arg *)p;
    for (;;) {
        pthread_barrier_wait(a->bar);          /* wait for thread 0 to post step j */
        int j = *a->jstep;
        if (j < 0) break;
        if (!*a->skip) {
            int ncols = a->n - (j + 1);
            int c0 = j + 1 + (int)((long)ncols * a->tid / a->nthreads);
            int c1 = j + 1 + (int)((long)ncols * (a->tid + 1) / a->nthreads);
            rank1_cols(a->A, a->lda, a->m, j, c0, c1);
        }
        pthread_barrier_wait(a->bar);          /* step j done */
    }
    return NULL;
}

/* Pivot choice of step j: first index of the largest |A(i, j)|, i = j..m-1.
 * A NaN has no magnitude and never wins a strict comparison, so it is never
 * chosen; a column with no other entry keeps p = j.  `gap` (optional)
 * receives (|p1| - |p2|) / |p1| for the two largest magnitudes, used to tell
 * true pivot disagreements from near-ties. */
static int pivot_of_column(const double *A, int lda, int m, int j, double *gap)
{
    int p = j;
    double best = -1.0, second = -1.0;
    for (int i = j; i < m; ++i) {
        double v = fabs(AT(A, lda, i, j));
        if (v > best) { second = best; best = v; p = i; }
        else if (v > second) second = v;
    }
    if (gap) *gap = (best > 0.0 && second >= 0.0) ? (best - second) / best : 1.0;
    return p;
}

/* oracle_getrf_forced: oracle_getrf in which the pivot of step j is row
 * forced[j] (0-based, j <= forced[j] < m) wherever forced != NULL and
 * forced[j] >= 0; every other step searches as usual.  It serves the near-tie
 * rule of the parity tests: when another implementation picks a different
 * pivot at a step whose top-2 gap is within rounding, the elimination is
 * re-run with that choice and compared from there on.  gaps[j] still reports
 * the search's own top-2 gap.  Returns -1 for a bad argument or a forced row
 * outside j..m-1 (A is then partly eliminated). */
int oracle_getrf_forced(int m, int n, double *A, int lda, int *ipiv, double *gaps, int nthreads,
                        const int *forced);

int oracle_getrf(int m, int n, double *A, int lda, int *ipiv, double *gaps, int nthreads)
{
    return oracle_getrf_forced(m, n, A, lda, ipiv, gaps, nthreads, NULL);
}

int oracle_getrf_forced(int m, int n, double *A, int lda, int *ipiv, double *gaps, int nthreads,
                        const int *forced)
{
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return -1;
    int info = 0;
    int kmax = m < n ? m : n;
    if (forced)
        for (int j = 0; j < kmax; ++j)
            if (forced[j] >= m || (forced[j] >= 0 && forced[j] < j)) return -1;
    if (nthreads < 1) nthreads = 1;
    pthread_barrier_t bar;
    pthread_t *th = NULL;
    upd_arg *args = NULL;
    volatile int jstep = 0, skip = 0;
    if (nthreads > 1) {
        pthread_barrier_init(&bar, NULL, (unsigned)nthreads);
        th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
        args = (upd_arg *)calloc((size_t)nthreads, sizeof(upd_arg));
        for (int t = 0; t < nthreads; ++t) {
            args[t] = (upd_arg){m, n, lda, A, nthreads, t, &bar, &jstep, &skip};
            if (t > 0) pthread_create(&th[t], NULL, upd_worker, &args[t]);
        }
    }
    for (int j = 0; j < kmax; ++j) {
        int p = pivot_of_column(A, lda, m, j, gaps ? &gaps[j] : NULL);
        if (forced && forced[j] >= 0) p = forced[j];
        ipiv[j] = p + 1;
        int zero = (AT(A, lda, p, j) == 0.0);
        if (zero) {
            if (info == 0) info = j + 1;
        } else {
            if (p != j)                                  /* interchange full rows */
                for (int c = 0; c < n; ++c) {
                    double t = AT(A, lda, j, c);
                    AT(A, lda, j, c) = AT(A, lda, p, c);
                    AT(A, lda, p, c) = t;
                }
            const double alpha = AT(A, lda, j, j);
            for (int i = j + 1; i < m; ++i)                /* rl1: divide, not multiply */
                AT(A, lda, i, j) = AT(A, lda, i, j) / alpha;
        }
        if (nthreads > 1) {
            jstep = j; skip = zero;
            pthread_barrier_wait(&bar);
            int ncols = n - (j + 1);
            if (!zero) rank1_cols(A, lda, m, j, j + 1, j + 1 + (int)((long)ncols / nthreads));
            pthread_barrier_wait(&bar);
        } else if (!zero) {
            rank1_cols(A, lda, m, j, j + 1, n);
        }
    }
    if (nthreads > 1) {
        jstep = -1;
        pthread_barrier_wait(&bar);
        for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
        pthread_barrier_destroy(&bar);
        free(th); free(args);
    }
    return info;
}

/* ------------------------------------------------------------------------ */
/* Solve A X = B with the factors of oracle_getrf (LAPACK getrs, no transpose):
 *   B := P B (interchanges in order j = 0..n-1), then
 *   L Y = B by forward substitution (unit diagonal), then
 *   U X = Y by back substitution.
 * Section 1 names the solution of linear systems as the use of the LU factors.
 * ------------------------------------------------------------------------ */
int oracle_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv, double *B, int ldb)
{
    if (n < 0 || nrhs < 0 || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1)) return -1;
    for (int r = 0; r < nrhs; ++r) {
        double *b = B + (size_t)r * (size_t)ldb;
        for (int j = 0; j < n; ++j) {
            int p = ipiv[j] - 1;
            if (p != j) { double t = b[j]; b[j] = b[p]; b[p] = t; }
        }
        for (int j = 0; j < n; ++j)                       /* L y = b */
            for (int i = j + 1; i < n; ++i)
                b[i] = b[i] - AT(LU, lda, i, j) * b[j];
        for (int j = n - 1; j >= 0; --j) {                /* U x = y */
            b[j] = b[j] / AT(LU, lda, j, j);
            for (int i = 0; i < j; ++i)
                b[i] = b[i] - AT(LU, lda, i, j) * b[j];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Checkers.
 * ------------------------------------------------------------------------ */

/* Apply the interchanges of ipiv (in order) to the rows of the m x n matrix X. */
void oracle_apply_pivots(int m, int n, double *X, int ldx, const int *ipiv, int k)
{
    for (int j = 0; j < k; ++j) {
        int p = ipiv[j] - 1;
        if (p == j) continue;
        for (int c = 0; c < n; ++c) {
            double t = AT(X, ldx, j, c);
            AT(X, ldx, j, c) = AT(X, ldx, p, c);
            AT(X, ldx, p, c) = t;
        }
    }
}

/* Frobenius norm of (P A - L U) and of A, computed directly (O(n^3)).
 * out[0] = ||PA - LU||_F, out[1] = ||A||_F. */
void oracle_lu_residual_fro(int n, const double *A, int lda, const double *LU, int ldlu,
                            const int *ipiv, double *out)
{
    double *PA = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) PA[i + (size_t)j * n] = AT(A, lda, i, j);
    oracle_apply_pivots(n, n, PA, n, ipiv, n);
    double r2 = 0.0, a2 = 0.0;
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            int kmax = i < j ? i : j;                    /* (L U)(i,j) = sum_{k<=min(i,j)} l_ik u_kj */
            for (int k = 0; k <= kmax; ++k) {
                double l = (k == i) ? 1.0 : AT(LU, ldlu, i, k);
                s += l * AT(LU, ldlu, k, j);
            }
            double d = PA[i + (size_t)j * n] - s;
            r2 += d * d;
            a2 += PA[i + (size_t)j * n] * PA[i + (size_t)j * n];
        }
    }
    free(PA);
    out[0] = sqrt(r2);
    out[1] = sqrt(a2);
}

/* Freivalds-style probe: out[0] = ||P A w - L (U w)||_2, out[1] = ||A||_F,
 * out[2] = ||w||_2.  O(n^2). */
void oracle_lu_residual_probe(int n, const double *A, int lda, const double *LU, int ldlu,
                              const int *ipiv, const double *w, double *out)
{
    double *t = (double *)calloc((size_t)n, sizeof(double));
    double *y = (double *)calloc((size_t)n, sizeof(double));
    double a2 = 0.0, w2 = 0.0;
    for (int i = 0; i < n; ++i) w2 += w[i] * w[i];
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double v = AT(A, lda, i, j);
            t[i] += v * w[j];
            a2 += v * v;
        }
    oracle_apply_pivots(n, 1, t, n, ipiv, n);            /* t = P A w */
    for (int j = 0; j < n; ++j)                           /* y = U w */
        for (int i = 0; i <= j; ++i) y[i] += AT(LU, ldlu, i, j) * w[j];
    double r2 = 0.0;
    for (int i = 0; i < n; ++i) {                         /* (L y)_i */
        double s = y[i];
        for (int k = 0; k < i; ++k) s += AT(LU, ldlu, i, k) * y[k];
        double d = t[i] - s;
        r2 += d * d;
    }
    free(t); free(y);
    out[0] = sqrt(r2); out[1] = sqrt(a2); out[2] = sqrt(w2);
}

/* Normwise backward error of a computed solution, per right-hand side r:
 *   eta_r = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
 * (Rigal and Gaches).  The residual is accumulated in FP64 in column order.
 * Returns max_r eta_r; eta[r] receives each value when eta != NULL. */
double oracle_backward_error(int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                             const double *B, int ldb, double *eta)
{
    double anorm = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += fabs(AT(A, lda, i, j));
        if (s > anorm) anorm = s;
    }
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        const double *x = X + (size_t)c * (size_t)ldx;
        const double *b = B + (size_t)c * (size_t)ldb;
        for (int i = 0; i < n; ++i) r[i] = b[i];
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) r[i] -= AT(A, lda, i, j) * x[j];
        double rn = 0.0, xn = 0.0, bn = 0.0;
        for (int i = 0; i < n; ++i) {
            if (fabs(r[i]) > rn) rn = fabs(r[i]);
            if (fabs(x[i]) > xn) xn = fabs(x[i]);
            if (fabs(b[i]) > bn) bn = fabs(b[i]);
        }
        double e = rn / (anorm * xn + bn);
        if (eta) eta[c] = e;
        if (e > worst) worst = e;
    }
    free(r);
    return worst;
}

/* Batched driver: factor and solve `count` independent matrices, one after the
 * other (each is exactly oracle_getrf + oracle_getrs).  Matrix t has order
 * ns[t], leading dimension ns[t], and starts at A + aoff[t]; its right-hand
 * side (length ns[t]) starts at B + boff[t]; its pivots at ipiv + poff[t]. */
void oracle_getrf_getrs_batched(int count, const int *ns, double *A, const long *aoff,
                                int *ipiv, const long *poff, double *B, const long *boff, int *info)
{
    for (int t = 0; t < count; ++t) {
        int n = ns[t];
        info[t] = oracle_getrf(n, n, A + aoff[t], n, ipiv + poff[t], NULL, 1);
        oracle_getrs(n, 1, A + aoff[t], n, ipiv + poff[t], B + boff[t], n);
    }
}

/* ------------------------------------------------------------------------ */
/* Unblocked right-looking Cholesky factorization A = L L^T of a symmetric
 * positive definite matrix (lower triangle referenced and overwritten; the
 * strictly upper part is not touched), the factorization the paper names as
 * the next case for the same scheme (section 1: the ideas carry over to other
 * dense factorizations).  For each column j:
 *   l_jj = sqrt(a_jj)                      (a_jj already updated)
 *   l_ij = a_ij / l_jj,  i > j             (division, not a reciprocal)
 *   a_ic = a_ic - l_ij * l_cj, j < c <= i  (lower triangle only, two roundings)
 * Returns 0, or j+1 for the first column whose updated diagonal entry is not
 * positive (LAPACK potrf's info; the factorization stops there), or -1 for a
 * bad argument.
 * ------------------------------------------------------------------------ */
int oracle_potrf(int n, double *A, int lda)
{
    if (n < 0 || lda < (n > 1 ? n : 1)) return -1;
    for (int j = 0; j < n; ++j) {
        const double d = AT(A, lda, j, j);
        if (!(d > 0.0)) return j + 1;
        const double l = sqrt(d);
        AT(A, lda, j, j) = l;
        for (int i = j + 1; i < n; ++i) AT(A, lda, i, j) = AT(A, lda, i, j) / l;
        for (int c = j + 1; c < n; ++c) {
            const double lc = AT(A, lda, c, j);
            for (int i = c; i < n; ++i)
                AT(A, lda, i, c) = AT(A, lda, i, c) - AT(A, lda, i, j) * lc;
        }
    }
    return 0;
}

/* Solve A X = B with the Cholesky factor L (lower): L Y = B, then L^T X = Y. */
int oracle_potrs(int n, int nrhs, const double *L, int lda, double *B, int ldb)
{
    if (n < 0 || nrhs < 0 || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1)) return -1;
    for (int r = 0; r < nrhs; ++r) {
        double *b = B + (size_t)r * (size_t)ldb;
        for (int j = 0; j < n; ++j) {                     /* L y = b */
            b[j] = b[j] / AT(L, lda, j, j);
            for (int i = j + 1; i < n; ++i) b[i] = b[i] - AT(L, lda, i, j) * b[j];
        }
        for (int j = n - 1; j >= 0; --j) {                /* L^T x = y */
            double s = b[j];
            for (int i = j + 1; i < n; ++i) s = s - AT(L, lda, i, j) * b[i];
            b[j] = s / AT(L, lda, j, j);
        }
    }
    return 0;
}
