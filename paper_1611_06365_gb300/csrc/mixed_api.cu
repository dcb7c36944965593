// lu_solve_mixed: FP32 LU with a (split-)BF16 tensor-core trailing update, recovered
// to FP64 accuracy by iterative refinement (not part of the paper: it refines
// the paper's blocked look-ahead factorization computed in lower precision).
//
// Ladder, in order, each rung entered only when the previous one stalls:
//   0  classic refinement: x += U^{-1} L^{-1} P r with r = b - A x in FP64;
//      if it stalls on the factors of a tensor-core update (BF16, split BF16,
//      FP8), the matrix is refactored once with the FP32 update and refined
//      on from the current x (report.f32_refactor = 1);
//   1  GMRES-IR (Carson and Higham, SIAM J. Sci. Comput. 39(6), 2017), here
//      in its flexible form: the correction equation A d = r is solved by
//      FGMRES (Saad, SIAM J. Sci. Comput. 14(2), 1993) with the FP32 factors
//      as right preconditioner and FP64 products with A, so that rounding in
//      the FP32 preconditioner solve does not limit the attainable accuracy;
//   2  the FP64 factorization of this library (by default with the emulated
//      FP64 update on the tensor cores), then classic refinement; if that
//      does not reach the target, the FP64 factorization with the DFMA update.
// Convergence: normwise backward error
//   eta = max_q ||b_q - A x_q||_inf / (||A||_inf ||x_q||_inf + ||b_q||_inf)
// at most `tol`.  Stall: eta has not halved over the last two steps, or
// max_iter steps were taken on the rung.
// Cost model (unless opts->fallback_ratio < 0): the FP64 fallback is
// predicted to cost C = ratio x (the first factorization's measured time),
// the ratio measured by the last fallback of the same order in this process
// or a default.  The low-precision rungs may spend at most C of refinement
// time before the fallback is taken (the rent-or-buy rule: the whole call
// then costs at most the factorization plus twice C), and a rung stops as
// soon as its own contraction predicts it would pass that budget: classic
// refinement from the observed ratio of successive backward errors, the FP32
// refactorization from its predicted cost, GMRES-IR from the time left.  With
// the cost model on, a condition estimate (one solve with the first factors and
// a random right-hand side) sends a matrix whose estimate times eps32 exceeds 16
// straight to the fallback once classic refinement stalls.
// Forward-error estimate: the correction one more refinement step would make,
// relative to the solution: max_q ||d_q||_inf / ||x_q||_inf with d = M^{-1} r,
// r = b - A x in FP64 and M the factors of the rung that finished (the
// estimate refinement offers for the error of its iterate: Demmel, Hida,
// Kahan, Li, Mukherjee and Riedy, "Error bounds from extra-precise iterative
// refinement", ACM TOMS 32(2), 2006).  It costs one residual and one solve;
// with FP32 factors it is as good as M^{-1} approximates A^{-1}.
#include "common.cuh"
#include <algorithm>
#include <chrono>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

using namespace lu;

namespace {

struct Buf {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Buf(cudaStream_t st) : s(st) {}
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        void *v = nullptr;
        cudaError_t e = cudaMallocAsync(&v, std::max<size_t>(count, 1) * sizeof(T), s);
        if (e != cudaSuccess) return e;
        ptrs.push_back(v);
        *p = static_cast<T *>(v);
        return cudaSuccess;
    }
    ~Buf() {
        for (void *v : ptrs) cudaFreeAsync(v, s);
    }
};

double bits_to_double(unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Measured cost ratios of this process, per (order, kind): kind 0 = FP64 fallback
// with the emulated update, 1 = with the DFMA update, 2 = FP32 refactorization;
// each relative to the first (tensor-core) factorization of the same call.
std::mutex g_ratio_mu;
std::map<std::pair<int, int>, double> g_ratio;

double ratio_get(int n, int kind, double dflt) {
    std::lock_guard<std::mutex> lk(g_ratio_mu);
    auto it = g_ratio.find({n, kind});
    return it == g_ratio.end() ? dflt : it->second;
}
void ratio_put(int n, int kind, double r) {
    if (!(r > 0.0) || !std::isfinite(r)) return;
    std::lock_guard<std::mutex> lk(g_ratio_mu);
    g_ratio[{n, kind}] = r;
}

}  // namespace

// max_q ||d_q||_inf / ||x_q||_inf from device norms (synchronizes s)
static int ferr_now(int nrhs, const unsigned long long *d_dmax, const unsigned long long *d_xmax, double *ferr,
                    cudaStream_t s) {
    std::vector<unsigned long long> h(2 * (size_t)nrhs);
    LU_CUDA_TRY(cudaMemcpyAsync(h.data(), d_dmax, sizeof(unsigned long long) * nrhs, cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaMemcpyAsync(h.data() + nrhs, d_xmax, sizeof(unsigned long long) * nrhs, cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaStreamSynchronize(s));
    double worst = 0.0;
    for (int q = 0; q < nrhs; ++q) {
        const double d = bits_to_double(h[q]), x = bits_to_double(h[nrhs + q]);
        double f = x > 0.0 ? d / x : (d > 0.0 ? INFINITY : 0.0);
        if (std::isnan(f)) f = INFINITY;
        worst = std::max(worst, f);
    }
    *ferr = worst;
    return LU_OK;
}

// eta for each column from device norms (synchronizes s)
static int eta_now(int nrhs, const unsigned long long *d_rmax, const unsigned long long *d_xmax, double anorm,
                   const std::vector<double> &bnorm, double *eta, cudaStream_t s) {
    std::vector<unsigned long long> h(2 * (size_t)nrhs);
    LU_CUDA_TRY(cudaMemcpyAsync(h.data(), d_rmax, sizeof(unsigned long long) * nrhs, cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaMemcpyAsync(h.data() + nrhs, d_xmax, sizeof(unsigned long long) * nrhs, cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaStreamSynchronize(s));
    double worst = 0.0;
    for (int q = 0; q < nrhs; ++q) {
        const double r = bits_to_double(h[q]), x = bits_to_double(h[nrhs + q]);
        const double den = anorm * x + bnorm[q];
        double e = den > 0.0 ? r / den : (r > 0.0 ? INFINITY : 0.0);
        if (std::isnan(e)) e = INFINITY;
        worst = std::max(worst, e);
    }
    *eta = worst;
    return LU_OK;
}

extern "C" int lu_solve_mixed(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb, double *dX, int ldx,
                              const lu_mixed_opts *opts, lu_mixed_report *rep, void *stream) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (n > 0 && !dA) return -3;
    if (lda < std::max(1, n)) return -4;
    if (n > 0 && nrhs > 0 && !dB) return -5;
    if (ldb < std::max(1, n)) return -6;
    if (n > 0 && nrhs > 0 && !dX) return -7;
    if (ldx < std::max(1, n)) return -8;
    if (opts && (opts->update != LU_UPDATE_NATIVE && opts->update != LU_UPDATE_BF16 && opts->update != LU_UPDATE_BF16X3 &&
                 opts->update != LU_UPDATE_FP8))
        return -9;
    if (opts && (opts->nb < 0 || opts->max_iter < 0 || opts->tol < 0 || opts->gmres_restart < 0)) return -9;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lu_mixed_report r = {};
    const int update = opts ? opts->update : LU_UPDATE_BF16X3;
    const int max_iter = (opts && opts->max_iter > 0) ? opts->max_iter : 30;
    const double tol = (opts && opts->tol > 0) ? opts->tol : 1e-14;
    const bool allow_gmres = opts ? opts->allow_gmres != 0 : true;
    const bool allow_fb = opts ? opts->allow_fallback != 0 : true;
    const int restart = (opts && opts->gmres_restart > 0) ? opts->gmres_restart : 30;
    const bool fp64_only = opts && opts->fp64_factor != 0;
    if (n == 0 || nrhs == 0) {
        if (rep) *rep = r;
        return LU_OK;
    }
    cudaEvent_t e0, e1, e2;
    LU_CUDA_TRY(cudaEventCreate(&e0));
    LU_CUDA_TRY(cudaEventCreate(&e1));
    LU_CUDA_TRY(cudaEventCreate(&e2));
    LU_CUDA_TRY(cudaEventRecord(e0, s));

    Buf ws(s);
    const int ld32 = (n + 31) & ~31;
    float *A32 = nullptr, *R32 = nullptr;
    int *ipiv = nullptr, *perm = nullptr, *info = nullptr;
    double *rowsum = nullptr, *R = nullptr, *part = nullptr;
    unsigned long long *norms = nullptr;   // [0] anorm, [1..nrhs] rmax, [1+nrhs..] xmax, [1+2nrhs..] bmax, [1+3nrhs..] dmax
    LU_CUDA_TRY(ws.get(&A32, (size_t)ld32 * n));
    LU_CUDA_TRY(ws.get(&R32, (size_t)n * nrhs));
    LU_CUDA_TRY(ws.get(&ipiv, n));
    LU_CUDA_TRY(ws.get(&perm, n));
    LU_CUDA_TRY(ws.get(&info, 1));
    LU_CUDA_TRY(ws.get(&rowsum, n));
    LU_CUDA_TRY(ws.get(&R, (size_t)n * nrhs));
    LU_CUDA_TRY(ws.get(&part, residual_workspace_doubles(n, nrhs)));
    LU_CUDA_TRY(ws.get(&norms, 1 + 4 * (size_t)nrhs));
    float *Dinv = nullptr;   // inverses of the FP32 factors' diagonal blocks (preconditioner solves)
    LU_CUDA_TRY(ws.get(&Dinv, f32_diag_inverse_elems(n)));
    unsigned long long *d_anorm = norms, *d_rmax = norms + 1, *d_xmax = norms + 1 + nrhs, *d_bmax = norms + 1 + 2 * nrhs;
    unsigned long long *d_dmax = norms + 1 + 3 * nrhs;

    // ||A||_inf and ||b||_inf
    LU_CUDA_TRY(launch_cast_rowsum(n, dA, lda, A32, ld32, rowsum, s));
    LU_CUDA_TRY(launch_vecmax(n, rowsum, d_anorm, s));
    LU_CUDA_TRY(launch_absmax(n, nrhs, dB, ldb, d_bmax, s));
    // FP32 factorization
    lu_opts fo = {};
    fo.update = update;
    fo.nb = opts ? opts->nb : 0;
    int rc = LU_OK;
    if (!fp64_only) {
        rc = factor_f32_internal(n, A32, ld32, ipiv, info, perm, &fo, s);
        if (rc != LU_OK) return rc;
        rc = f32_diag_inverse(n, A32, ld32, Dinv, s);
        if (rc != LU_OK) return rc;
    } else {
        LU_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
    }
    LU_CUDA_TRY(cudaEventRecord(e1, s));
    std::vector<unsigned long long> hn(1 + 3 * (size_t)nrhs);
    int hinfo = 0;
    LU_CUDA_TRY(cudaMemcpyAsync(hn.data(), norms, sizeof(unsigned long long) * hn.size(), cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaStreamSynchronize(s));
    r.info = hinfo;
    // cost model: the predicted cost of the FP64 fallback, the budget of the rungs before it
    float tf_ms = 0.f;
    LU_CUDA_TRY(cudaEventElapsedTime(&tf_ms, e0, e1));
    const bool fb_native = opts && opts->fallback_native;
    const bool cost_on = !(opts && opts->fallback_ratio < 0) && allow_fb && !fp64_only && tf_ms > 0.f;
    const double ratio64 = (opts && opts->fallback_ratio > 0) ? opts->fallback_ratio
                                                              : ratio_get(n, fb_native ? 1 : 0, fb_native ? 32.0 : 4.0);
    const double c64 = ratio64 * tf_ms;
    const auto t_ref = std::chrono::steady_clock::now();
    const char *log_env = getenv("LU_MIXED_LOG");
    const bool log_on = log_env && log_env[0] == '1';
    if (log_on)
        fprintf(stderr, "lu_solve_mixed: n %d nrhs %d factor %.2f ms, fallback predicted %.2f ms (ratio %.2f)\n", n, nrhs,
                tf_ms, c64, ratio64);
    const double anorm = bits_to_double(hn[0]);
    std::vector<double> bnorm(nrhs);
    for (int q = 0; q < nrhs; ++q) bnorm[q] = bits_to_double(hn[1 + 2 * nrhs + q]);
    // condition estimate: one solve with the first factors and a random right-hand side
    if (!fp64_only && hinfo == 0) {
        LU_CUDA_TRY(launch_fill_probe(n, 20161106ull + (unsigned long long)n, R32, s));
        rc = solve_f32_perm(n, 1, A32, ld32, perm, R32, n, s, Dinv);
        if (rc != LU_OK) return rc;
        unsigned long long *kbuf = nullptr;   // [0] = 0: scale 1; [1]: max |M^{-1} r|
        LU_CUDA_TRY(ws.get(&kbuf, 2));
        LU_CUDA_TRY(cudaMemsetAsync(kbuf, 0, 2 * sizeof(unsigned long long), s));
        LU_CUDA_TRY(launch_absmax_scaled_f32(n, 1, R32, n, kbuf, kbuf + 1, s));
        unsigned long long hk = 0;
        LU_CUDA_TRY(cudaMemcpyAsync(&hk, kbuf + 1, sizeof(hk), cudaMemcpyDeviceToHost, s));
        LU_CUDA_TRY(cudaStreamSynchronize(s));
        r.cond_est = anorm * bits_to_double(hk);   // ||r||_inf is 1 to within 2 / n
        if (log_on) fprintf(stderr, "lu_solve_mixed: condition estimate %.3e\n", r.cond_est);
    }

    // rung 0: classic refinement from x = 0, r = b
    LU_CUDA_TRY(cudaMemset2DAsync(dX, sizeof(double) * ldx, 0, sizeof(double) * n, nrhs, s));
    LU_CUDA_TRY(cudaMemcpy2DAsync(R, sizeof(double) * n, dB, sizeof(double) * ldb, sizeof(double) * n, nrhs,
                                  cudaMemcpyDeviceToDevice, s));
    LU_CUDA_TRY(cudaMemcpyAsync(d_rmax, d_bmax, sizeof(unsigned long long) * nrhs, cudaMemcpyDeviceToDevice, s));
    double eta = 1.0, ferr = INFINITY;
    bool factors64 = false;
    double *A64 = nullptr;
    double *Dinv64 = nullptr;   // inverses of the FP64 factors' diagonal blocks (refinement solves)
    int *perm64 = nullptr;
    std::vector<double> hist;
    bool done = false;
    // classic refinement with the FP32 factors in A32, from the current X and R
    auto classic = [&]() -> int {
        hist.clear();
        const auto t_rung = std::chrono::steady_clock::now();
        for (int it = 0; it < max_iter; ++it) {
            LU_CUDA_TRY(launch_to_f32_scaled(n, nrhs, R, n, d_rmax, R32, n, s));
            int rc2 = solve_f32_perm(n, nrhs, A32, ld32, perm, R32, n, s, Dinv);
            if (rc2 != LU_OK) return rc2;
            if (log_on) LU_CUDA_TRY(launch_absmax_scaled_f32(n, nrhs, R32, n, d_rmax, d_dmax, s));
            LU_CUDA_TRY(launch_axpy_scaled(n, nrhs, R32, n, d_rmax, dX, ldx, s));
            LU_CUDA_TRY(launch_residual(n, nrhs, dA, lda, dX, ldx, dB, ldb, R, n, part, d_rmax, s));
            LU_CUDA_TRY(launch_absmax(n, nrhs, dX, ldx, d_xmax, s));
            rc2 = eta_now(nrhs, d_rmax, d_xmax, anorm, bnorm, &eta, s);
            if (rc2 != LU_OK) return rc2;
            r.iterations++;
            hist.push_back(eta);
            if (log_on) {
                double corr = 0.0;   // max_q ||d_q|| / ||x_q|| of this step's correction
                rc2 = ferr_now(nrhs, d_dmax, d_xmax, &corr, s);
                if (rc2 != LU_OK) return rc2;
                fprintf(stderr, "lu_solve_mixed: classic step %d eta %.3e correction %.3e at %.2f ms\n", it, eta, corr,
                        ms_since(t_ref));
            }
            if (eta <= tol) { done = true; break; }
            const size_t h = hist.size();
            if (h >= 3 && !(hist[h - 1] <= 0.5 * hist[h - 3])) break;   // stalled
            const double rho = h >= 2 ? hist[h - 1] / hist[h - 2] : 1.0;
            if (cost_on && rho > 0.0 && rho < 1.0) {
                // steps still needed at the last contraction rate, at this rung's time per step
                // (no contraction is left to the stall rule)
                const double need = std::ceil(std::log(tol / eta) / std::log(rho));
                if (ms_since(t_ref) + need * ms_since(t_rung) / (it + 1) > c64) {
                    r.cost_stop = 1;
                    break;
                }
            }
        }
        return LU_OK;
    };
    // too ill-conditioned for FP32 factors: when the estimate times eps32 passes 16, no
    // low-precision rung is tried (measured at
    // n = 16384 on products of Householder reflectors: the estimate is 17 to 130 times
    // kappa_2; kappa_2 = 1e5 gives 1.5 and converges through the refactorization and GMRES-IR,
    // kappa_2 = 1e8 gives 199 and does not)
    const double cond_meter = r.cond_est * (double)FLT_EPSILON;
    const bool hopeless = cost_on && !fp64_only && hinfo == 0 && cond_meter > 16.0;
    if (hopeless) {
        r.cost_stop = 1;
        if (log_on) fprintf(stderr, "lu_solve_mixed: condition estimate x eps32 = %.3g: straight to FP64\n", cond_meter);
    }
    if (hinfo == 0 && !fp64_only && !hopeless) {
        rc = classic();
        if (rc != LU_OK) return rc;
    }
    // rung 0, second part: factors of the tensor-core update too coarse for this
    // matrix (refinement stalled) -- refactor with the FP32 update (FP32-accurate
    // factors) and refine on from the current solution
    const bool refactor_ok = !done && !fp64_only && !hopeless && update != LU_UPDATE_NATIVE && !(opts && opts->f32_refactor < 0);
    // the refactorization's own predicted cost decides (a classic rung the cost model
    // ended early is no reason to skip it: FP32 factors may contract where these did not)
    const bool refactor_too_dear = refactor_ok && cost_on && ms_since(t_ref) + ratio_get(n, 2, 1.5) * tf_ms >= c64;
    if (refactor_too_dear) r.cost_stop = 1;
    if (refactor_ok && !refactor_too_dear) {
        r.f32_refactor = 1;
        const auto t_rf = std::chrono::steady_clock::now();
        LU_CUDA_TRY(launch_cast_rowsum(n, dA, lda, A32, ld32, rowsum, s));
        lu_opts fo2 = {};
        fo2.update = LU_UPDATE_NATIVE;
        rc = factor_f32_internal(n, A32, ld32, ipiv, info, perm, &fo2, s);
        if (rc != LU_OK) return rc;
        rc = f32_diag_inverse(n, A32, ld32, Dinv, s);
        if (rc != LU_OK) return rc;
        LU_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
        LU_CUDA_TRY(cudaStreamSynchronize(s));
        if (tf_ms > 0.f) ratio_put(n, 2, ms_since(t_rf) / tf_ms);
        if (log_on) fprintf(stderr, "lu_solve_mixed: FP32 refactorization %.2f ms\n", ms_since(t_rf));
        if (hinfo == 0) {
            rc = classic();
            if (rc != LU_OK) return rc;
        }
    }
    // rung 1: GMRES-IR with the FP32 factors as preconditioner
    const double gm_budget = cost_on ? c64 - ms_since(t_ref) : 0.0;
    if (!done && hinfo == 0 && allow_gmres && !fp64_only && cost_on && gm_budget <= 0.0) r.cost_stop = 1;
    if (!done && hinfo == 0 && allow_gmres && !fp64_only && !hopeless && !(cost_on && gm_budget <= 0.0)) {
        r.rung = 1;
        int outer = 0, inner = 0;
        rc = gmres_ir(n, nrhs, dA, lda, dB, ldb, dX, ldx, A32, ld32, perm, anorm, bnorm.data(), tol, max_iter, restart, &outer,
                      &inner, &eta, s, cost_on ? gm_budget : 0.0, Dinv);
        if (rc != LU_OK) return rc;
        r.iterations += outer;
        r.gmres_iters += inner;
        done = eta <= tol;
        if (log_on)
            fprintf(stderr, "lu_solve_mixed: GMRES-IR %d outer %d inner, eta %.3e at %.2f ms (budget %.2f)\n", outer, inner,
                    eta, ms_since(t_ref), gm_budget);
        if (!done) {
            if (cost_on && ms_since(t_ref) >= c64) r.cost_stop = 1;
            // the iterate as it stands (a budget stop leaves columns unmeasured)
            LU_CUDA_TRY(launch_residual(n, nrhs, dA, lda, dX, ldx, dB, ldb, R, n, part, d_rmax, s));
            LU_CUDA_TRY(launch_absmax(n, nrhs, dX, ldx, d_xmax, s));
            rc = eta_now(nrhs, d_rmax, d_xmax, anorm, bnorm, &eta, s);
            if (rc != LU_OK) return rc;
            done = eta <= tol;
        }
    }
    // rung 2: FP64 factorization
    if (!done && (allow_fb || fp64_only)) {
        r.rung = 2;
        r.fell_back = fp64_only ? 0 : 1;
        const auto t_fb = std::chrono::steady_clock::now();
        int *ipiv64 = nullptr, *info64 = nullptr;
        factors64 = true;
        LU_CUDA_TRY(ws.get(&A64, (size_t)n * n));
        LU_CUDA_TRY(ws.get(&ipiv64, n));
        LU_CUDA_TRY(ws.get(&perm64, n));
        LU_CUDA_TRY(ws.get(&info64, 1));
        LU_CUDA_TRY(cudaMemcpy2DAsync(A64, sizeof(double) * n, dA, sizeof(double) * lda, sizeof(double) * n, n,
                                      cudaMemcpyDeviceToDevice, s));
        lu_opts o64 = {};
        o64.update = (opts && opts->fallback_native) ? LU_UPDATE_NATIVE : LU_UPDATE_F64EMU;
        rc = factor_f64_internal(n, A64, n, ipiv64, info64, perm64, &o64, s);
        if (rc != LU_OK) return rc;
        if (!Dinv64) LU_CUDA_TRY(ws.get(&Dinv64, f64_diag_inverse_elems(n)));
        rc = f64_diag_inverse(n, A64, n, Dinv64, s);
        if (rc != LU_OK) return rc;
        LU_CUDA_TRY(cudaMemset2DAsync(dX, sizeof(double) * ldx, 0, sizeof(double) * n, nrhs, s));
        LU_CUDA_TRY(cudaMemcpy2DAsync(R, sizeof(double) * n, dB, sizeof(double) * ldb, sizeof(double) * n, nrhs,
                                      cudaMemcpyDeviceToDevice, s));
        double *D = nullptr;
        LU_CUDA_TRY(ws.get(&D, (size_t)n * nrhs));
        // up to five refinement steps from the current X and R with the FP64 factors; the
        // solves use the diagonal-block inverses, and if that does not reach the target
        // (a diagonal block too ill-conditioned for its explicit inverse) exact substitution
        // takes over on the same factors
        auto refine64 = [&](const double *dinv) -> int {
            for (int it = 0; it < 5 && !(eta <= tol); ++it) {
                LU_CUDA_TRY(cudaMemcpyAsync(D, R, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, s));
                int rc2 = solve_f64_perm(n, nrhs, A64, n, perm64, D, n, s, dinv);
                if (rc2 != LU_OK) return rc2;
                LU_CUDA_TRY(launch_axpy_f64(n, nrhs, D, n, dX, ldx, s));   // X += D
                LU_CUDA_TRY(launch_residual(n, nrhs, dA, lda, dX, ldx, dB, ldb, R, n, part, d_rmax, s));
                LU_CUDA_TRY(launch_absmax(n, nrhs, dX, ldx, d_xmax, s));
                rc2 = eta_now(nrhs, d_rmax, d_xmax, anorm, bnorm, &eta, s);
                if (rc2 != LU_OK) return rc2;
                r.iterations++;
            }
            return LU_OK;
        };
        eta = INFINITY;
        if ((rc = refine64(Dinv64)) != LU_OK) return rc;
        if (!(eta <= tol) && (rc = refine64(nullptr)) != LU_OK) return rc;
        done = eta <= tol;
        if (!done && o64.update == LU_UPDATE_F64EMU && (allow_fb || fp64_only)) {
            // the emulated FP64 factors did not reach the target: the DFMA factorization
            LU_CUDA_TRY(cudaMemcpy2DAsync(A64, sizeof(double) * n, dA, sizeof(double) * lda, sizeof(double) * n, n,
                                          cudaMemcpyDeviceToDevice, s));
            o64.update = LU_UPDATE_NATIVE;
            rc = factor_f64_internal(n, A64, n, ipiv64, info64, perm64, &o64, s);
            if (rc != LU_OK) return rc;
            if (!Dinv64) LU_CUDA_TRY(ws.get(&Dinv64, f64_diag_inverse_elems(n)));
            rc = f64_diag_inverse(n, A64, n, Dinv64, s);
            if (rc != LU_OK) return rc;
            LU_CUDA_TRY(cudaMemset2DAsync(dX, sizeof(double) * ldx, 0, sizeof(double) * n, nrhs, s));
            LU_CUDA_TRY(cudaMemcpy2DAsync(R, sizeof(double) * n, dB, sizeof(double) * ldb, sizeof(double) * n, nrhs,
                                          cudaMemcpyDeviceToDevice, s));
            eta = INFINITY;
            if ((rc = refine64(Dinv64)) != LU_OK) return rc;
            if (!(eta <= tol) && (rc = refine64(nullptr)) != LU_OK) return rc;
            done = eta <= tol;
        }
        r.t_fallback_ms = ms_since(t_fb);
        if (log_on) fprintf(stderr, "lu_solve_mixed: FP64 fallback %.2f ms, eta %.3e\n", r.t_fallback_ms, eta);
        // learn the ratio of the fallback as asked for (not of one that needed the DFMA safety net)
        if (!fp64_only && tf_ms > 0.f && (fb_native || o64.update == LU_UPDATE_F64EMU))
            ratio_put(n, fb_native ? 1 : 0, r.t_fallback_ms / tf_ms);
    }
    // forward-error estimate: one more correction with the finishing rung's factors
    if (hinfo == 0 || factors64) {
        LU_CUDA_TRY(launch_residual(n, nrhs, dA, lda, dX, ldx, dB, ldb, R, n, part, d_rmax, s));
        LU_CUDA_TRY(launch_absmax(n, nrhs, dX, ldx, d_xmax, s));
        if (factors64) {
            double *D = nullptr;
            LU_CUDA_TRY(ws.get(&D, (size_t)n * nrhs));
            LU_CUDA_TRY(cudaMemcpyAsync(D, R, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, s));
            rc = solve_f64_perm(n, nrhs, A64, n, perm64, D, n, s, Dinv64);
            if (rc != LU_OK) return rc;
            LU_CUDA_TRY(launch_absmax(n, nrhs, D, n, d_dmax, s));
        } else {
            LU_CUDA_TRY(launch_to_f32_scaled(n, nrhs, R, n, d_rmax, R32, n, s));
            rc = solve_f32_perm(n, nrhs, A32, ld32, perm, R32, n, s, Dinv);
            if (rc != LU_OK) return rc;
            LU_CUDA_TRY(launch_absmax_scaled_f32(n, nrhs, R32, n, d_rmax, d_dmax, s));
        }
        rc = ferr_now(nrhs, d_dmax, d_xmax, &ferr, s);
        if (rc != LU_OK) return rc;
    }
    LU_CUDA_TRY(cudaEventRecord(e2, s));
    LU_CUDA_TRY(cudaEventSynchronize(e2));
    float t01 = 0, t12 = 0;
    cudaEventElapsedTime(&t01, e0, e1);
    cudaEventElapsedTime(&t12, e1, e2);
    r.t_factor_ms = t01;
    r.t_refine_ms = t12;
    r.t_total_ms = (double)t01 + t12;
    r.backward_error = eta;
    r.forward_error_est = ferr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (rep) *rep = r;
    return LU_OK;
}
