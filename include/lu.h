/*
 * lu.h -- C ABI of the GB300 LU-with-partial-pivoting library (liblu.so).
 *
 * The method: blocked right-looking LU factorization with partial pivoting,
 * P A = L U (section 3 of arXiv:1611.06365, "A Case for Malleable Thread-Level
 * Linear Algebra Libraries"), with static look-ahead (section 3.2, Figure 3,
 * equation (2x2)) whose panel resources rejoin the trailing update once the
 * next panel is factored (worker sharing, section 4.1).  On the GPU the panel
 * is one thread-block cluster and the update is a tile grid on a lower
 * priority stream; the hardware CTA scheduler hands the SMs freed by the panel
 * to the pending update tiles.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are column-major: element (i, j) of a matrix with leading
 *    dimension ld sits at offset i + j*ld (elements, not bytes).  ld >= max(1,n).
 *  - All matrix, vector, pivot and info pointers are DEVICE pointers owned by
 *    the caller, unless the argument is documented as host memory.  The
 *    library never frees caller memory.  Internal workspace is allocated
 *    stream-ordered (cudaMallocAsync) on the caller's stream and released
 *    before the call returns its work to that stream.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous with respect to the host unless stated otherwise; the work
 *    is ordered after prior work on `stream`, and later work on `stream` sees
 *    its results.
 *  - Pivots: int32, 1-based, LAPACK sequential-interchange meaning: at step j
 *    row j was interchanged with row ipiv[j]-1 (ipiv[j]-1 >= j).  Ties in the
 *    pivot search go to the smallest row index.
 *  - Return value: 0 on success; -i when argument i (1-based) is invalid
 *    (nothing is launched); LU_ERR_* (< -99) for runtime failures.
 *  - Numerical singularity is not an error: *info (device int) receives 0, or
 *    j > 0 when U(j,j) (1-based) is exactly zero for the first such j; the
 *    factorization is completed as LAPACK's getrf does (no interchange and no
 *    scaling for that column).
 *  - Every device-side wait between CTAs is bounded; when a bound expires the
 *    kernel records LU_ERR_TIMEOUT in a library status word (see
 *    lu_last_device_status) and returns instead of hanging.
 *  - The library keeps per-device state created on first use (two streams,
 *    events, the status word, the device address of lu_solve_noalloc's
 *    scratch array).  cudaDeviceReset destroys the context that state lives
 *    in: after a reset, unload and reload the library before calling it on
 *    that device again.
 */
#ifndef GB300_LU_H
#define GB300_LU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { LU_F64 = 0, LU_F32 = 1 } lu_dtype;

enum {
    LU_OK = 0,
    LU_ERR_CUDA = -100,        /* a CUDA runtime call failed */
    LU_ERR_NOMEM = -101,       /* workspace allocation failed */
    LU_ERR_TIMEOUT = -102,     /* a bounded device-side wait expired */
    LU_ERR_UNSUPPORTED = -103, /* valid request this build cannot serve */
    LU_ERR_SCRATCH = -104      /* request larger than the fixed scratch of lu_solve_noalloc */
};

/* Trailing-update arithmetic (LU_UPDATE_BF16 .. LU_UPDATE_FP8 for LU_F32
 * factorizations, LU_UPDATE_F64EMU for LU_F64). */
enum {
    LU_UPDATE_NATIVE = 0,  /* same precision as the storage (FP64 / FP32 SIMT) */
    LU_UPDATE_BF16 = 1,    /* BF16 operands on tcgen05 tensor cores, FP32 accumulate */
    LU_UPDATE_BF16X3 = 2,  /* split BF16 on tcgen05: x = hi + lo, three products
                              hi*hi + hi*lo + lo*hi per pair, FP32 accumulate
                              (about 16 significant bits per product) */
    LU_UPDATE_FP8 = 3,     /* FP8 e4m3 on tcgen05 (kind::f8f6f4), FP32 accumulate;
                              each staged row of L21 and column of U12 is
                              multiplied by the power of two that brings its
                              largest magnitude into (224, 448], and the
                              epilogue applies the exact inverse factors */
    LU_UPDATE_F64EMU = 4   /* FP64 emulated on tcgen05 BF16 tensor cores (LU_F64 only;
                              outer width b_o <= 64): every row of L21 and column of
                              U12 is split below a power-of-two scale into seven
                              8-bit BF16 digits (Ozaki, Ogita, Oishi and Rump,
                              Numer. Algorithms 59, 2012); the 28 digit products
                              that reach 2^-56 of the leading one are accumulated in
                              FP32 per diagonal (exactly for the five leading
                              diagonals, the last two sharing a rounded sum), added
                              exactly as a 64-bit integer and subtracted from C with
                              one FP64 rounding */
};

/* Tuning knobs.  Pass NULL for the built-in choice; a zero field means "auto". */
typedef struct {
    int nb;            /* outer panel width b_o (the algorithmic block size of section 3.1);
                          0 = LU_F64: 32 up to n = 8192, 64 beyond; LU_F32: 128 (SIMT
                          update) or 64 (tensor-core updates, 128 from n = 24576) */
    int nb_inner;      /* inner panel width b_i (section 4.2, outer vs inner LU) */
    int panel_ctas;    /* CTAs in the panel cluster, 1..16 (team PF size, section 3.2);
                          0 = 8 for LU_F64, 16 for LU_F32; a panel whose rows do not fit
                          that many CTAs' register tiles takes more */
    int lookahead;     /* 0 (auto) or 1: static look-ahead with worker sharing;
                          d = 2..4: look-ahead of depth d (the panel branch keeps the
                          next d column strips current, so panel k+1 no longer waits
                          for the remainder update of step k-1; section 3.2 notes the
                          look-ahead can span more than one panel);
                          -1: plain blocked RL without look-ahead */
    int update;        /* LU_UPDATE_*: BF16 .. FP8 with LU_F32, F64EMU with LU_F64 */
    long long spin_ns; /* bound for device-side waits in ns (0 = 2 s) */
    int update_ctas;   /* tensor-core updates (LU_F32 BF16 .. FP8, LU_F64 F64EMU): persistent
                          CTAs of the remainder update RU2 (section 3.2's split of the threads
                          between the panel and the update); 0 = one per SM */
    int sm_share;      /* tensor-core updates with look-ahead: 0 (default) or 1 = worker
                          sharing (section 4.1) between the panel and the persistent RU2:
                          RU2's CTAs on the SMs of one panel-cluster placement stop taking
                          tiles while panel k+1 waits for them, and a grid of as many CTAs
                          joins RU2's tile queue when the panel ends; -1 = off (RU2 keeps
                          its SMs until its queue is empty) */
    int tile;          /* trailing-update tile shape: 0 = auto; 1 = large (DFMA update 64 x 64
                          output tiles; emulated FP64 update tasks of 8 sub-tiles of 32 columns);
                          2 = small (32 x 32; 2 sub-tiles).  Changes the schedule, not the
                          arithmetic (results are the same bits); the FP32 tensor-core updates
                          have one shape and ignore it */
    int early_term;    /* early termination (section 4.2, Figure LU_LA_ET): 0 = off (default);
                          1 = the panel factorization of step k+1 stops at the end of the
                          inner panel during which the remainder update of step k finished,
                          and step k+1 then has the width the panel reached (an adaptive
                          b_o); 2 = stop at the end of the first inner panel of every panel
                          (a fixed schedule through the same path, for tests).  Takes effect
                          when the inner width is below the outer one (nb_inner < nb) and
                          needs look-ahead of depth 1 (lookahead 0 or 1).  The host learns
                          each panel's width before enqueueing the next step: lu_factor then
                          returns after the last panel has run, and a stream under capture
                          is refused (LU_ERR_UNSUPPORTED).  The pivots follow the unblocked
                          algorithm as always; the rounding of the factors depends on where
                          the panels stopped.  lu_last_panel_widths reports the widths. */
} lu_opts;

/*
 * lu_factor -- P A = L U of the n x n matrix A, in place.
 *   Section 3.1, Figure 1 (right), blocked right-looking LU: per panel of b
 *   columns, RL1 panel LU with partial pivoting, the panel's interchanges
 *   applied to the other columns, RL2 A12 := trilu(A11)^{-1} A12, RL3
 *   A22 := A22 - A21 A12; with look-ahead (section 3.2, Figure 3) unless
 *   opts->lookahead == -1.
 *   dt    LU_F64 (dA is double*) or LU_F32 (dA is float*).
 *   n     order, n >= 0.               dA    device, n x n, leading dim lda.
 *   lda   >= max(1, n).                d_ipiv device int[n] (output).
 *   d_info device int (output).        opts  host pointer or NULL; NULL
 *   or a zero field takes the autotuner's entry for this order (lu_autotune
 *   below), else the built-in choice.
 *   On return A holds L (strictly lower, unit diagonal implied) and U.
 */
int lu_factor(lu_dtype dt, int n, void *dA, int lda, int *d_ipiv, int *d_info,
              const lu_opts *opts, void *stream);

/*
 * lu_last_panel_widths -- the widths of the panels of the last LU
 *   factorization enqueued on the current device (lu_factor, or the one inside
 *   lu_solve_mixed), in order: all b_o but the last unless early termination
 *   shortened some (section 4.2).  Copies min(count, cap) of them to the host
 *   array `widths` (may be NULL when cap = 0) and returns count, or -1 when no
 *   factorization ran on this device yet.  Host-side bookkeeping: no CUDA work.
 */
int lu_last_panel_widths(int *widths, int cap);

/*
 * lu_solve -- X := A^{-1} B with the factors from lu_factor (no transpose).
 *   Applies the interchanges of ipiv to B in order, then L Y = P B (unit
 *   lower) and U X = Y (upper).  Section 1 names linear systems as the use of
 *   the factorization.
 *   dLU   device factors (lda).  dB device n x nrhs (ldb), overwritten by X.
 *   nrhs >= 0.  A zero U(j,j) yields Inf/NaN, as in LAPACK.
 */
int lu_solve(lu_dtype dt, int n, int nrhs, const void *dLU, int lda, const int *d_ipiv,
             void *dB, int ldb, void *stream);

/*
 * lu_solve_noalloc -- lu_solve that allocates no memory.  (No counterpart in
 * the paper: it exists for callers that cannot allocate device memory during
 * a solve, e.g. an application whose framework has reserved the device
 * memory for its own pool, so any cudaMalloc would fail, or a latency-critical
 * loop that cannot afford an allocation that may wait for the device.)
 *   Arguments as lu_solve; d_status (device int, may be NULL) receives
 *   LU_OK, or LU_ERR_TIMEOUT if a bounded wait of the substitution expired.
 *   Workspace comes from one fixed array in device memory of
 *   lu_solve_noalloc_capacity() bytes (4 MiB) that every GPU loading the
 *   library keeps until exit.  A request needs about
 *   4 n + elem * n * nrhs + 16 n min(nrhs, 16) + 256 bytes plus alignment
 *   (elem = 8 for LU_F64, 4 for LU_F32; e.g. n = 65536, nrhs = 1 in FP32
 *   takes 1.5 MiB); a larger one returns LU_ERR_SCRATCH and launches
 *   nothing.  The first call on a device looks up the array's device address
 *   (make it before any stream capture).  All calls share the array: calls
 *   whose work overlaps on the GPU race and must be serialized by the caller.
 */
int lu_solve_noalloc(lu_dtype dt, int n, int nrhs, const void *dLU, int lda, const int *d_ipiv,
                     void *dB, int ldb, int *d_status, void *stream);
size_t lu_solve_noalloc_capacity(void);

/*
 * lu_factor_batched -- lu_factor applied to `batch` independent matrices of
 * possibly different orders in ONE factorization launch.
 *   d_n    device int[batch], orders (0 <= n_t <= max_n).
 *   d_A    device array of device pointers, matrix t in column-major.
 *   d_lda  device int[batch] (lda_t >= max(1, n_t)).
 *   d_ipiv device array of device int* (n_t entries each).
 *   d_info device int[batch].
 *   max_n  host int, >= every n_t; at most 1024.
 *   opts   NULL or opts->nb: 0 = automatic; 16 or 32 = the blocked kernel
 *          with that panel width (max_n <= 256; section 3.1, Figure 1 right:
 *          persistent CTAs take matrices largest first from a queue, panel
 *          rows in registers, U12 solve and trailing update on chip);
 *          1 = the unblocked kernel (Figure 1 left, one CTA per matrix, the
 *          only one for max_n > 256).  Other values return -9.  Both kernels
 *          apply the same fused multiply-adds in the same order to every
 *          element, so their factors and pivots are identical.
 *   The blocked kernel allocates a small stream-ordered workspace (the queue
 *   and the size order, 4 (batch + 32) bytes).
 */
int lu_factor_batched(lu_dtype dt, int batch, const int *d_n, void *const *d_A, const int *d_lda,
                      int *const *d_ipiv, int *d_info, int max_n, const lu_opts *opts, void *stream);

/*
 * lu_solve_batched -- lu_solve for each member of a batch, nrhs right-hand
 * sides each (max_n <= 256: one warp per matrix and right-hand side; larger:
 * one CTA per matrix).  d_B: device array of device pointers, d_ldb device
 * int[batch].
 */
int lu_solve_batched(lu_dtype dt, int batch, int nrhs, const int *d_n, const void *const *d_LU,
                     const int *d_lda, const int *const *d_ipiv, void *const *d_B, const int *d_ldb,
                     int max_n, void *stream);

/* Options of the mixed-precision solver.  NULL selects: split-BF16 update, auto nb,
 * 30 iterations, tol 1e-14, GMRES-IR and FP64 fallback both enabled, no
 * fp64_factor, the FP64 factorization with the emulated FP64 update. */
typedef struct {
    int update;          /* LU_UPDATE_BF16X3 (default), LU_UPDATE_BF16, LU_UPDATE_FP8 or
                            LU_UPDATE_NATIVE (FP32) */
    int nb;              /* outer panel width for the FP32 factorization (0 = auto) */
    int max_iter;        /* refinement iterations before declaring a stall (0 = 30) */
    double tol;          /* target normwise backward error (0 = 1e-14) */
    int allow_gmres;     /* 1 enables GMRES-IR when classic refinement stalls */
    int allow_fallback;  /* 1 enables the FP64 factorization when refinement stalls */
    int gmres_restart;   /* Krylov dimension of GMRES-IR (0 = 30) */
    int fp64_factor;     /* 1: skip the low-precision rungs and factor in FP64 (the
                            FP64 path measured the same way, for comparison) */
    int fallback_native; /* FP64 factorization of rung 2 (and of fp64_factor): 0 = with the
                            emulated FP64 update (LU_UPDATE_F64EMU), 1 = with the plain
                            DFMA update (LU_UPDATE_NATIVE) */
    int f32_refactor;    /* 0: when classic refinement stalls on the factors of a tensor-core
                            update, refactor once with the FP32 update and refine on before
                            GMRES-IR; -1: never */
    double fallback_ratio; /* cost model of the ladder: the FP64 fallback (factorization and
                            refinement) is predicted to take fallback_ratio times the first
                            factorization's measured time; 0 = the ratio measured by an earlier
                            fallback of the same order in this process, else 4 (emulated FP64
                            update) or 32 (DFMA update); < 0 = no cost model.  With the model
                            on, a matrix whose condition estimate (report.cond_est) times
                            eps32 exceeds 16 goes to the fallback as soon as classic
                            refinement stalls */
} lu_mixed_opts;

/* Result of lu_solve_mixed (host memory, filled before the call returns). */
typedef struct {
    int rung;            /* 0 classic IR, 1 GMRES-IR, 2 FP64 factorization fallback */
    int iterations;      /* refinement steps taken (all rungs) */
    int gmres_iters;     /* total inner GMRES iterations */
    int fell_back;       /* 1 if the FP64 factorization was used */
    int info;            /* info of the FP32 factorization (0 = nonsingular) */
    double backward_error;  /* final max_r ||b-Ax||_inf/(||A||_inf ||x||_inf + ||b||_inf) */
    double t_factor_ms;  /* device time of the FP32 factorization */
    double t_refine_ms;  /* device time of refinement (and fallback) */
    double t_total_ms;   /* device time of the whole call */
    double forward_error_est;  /* estimate of max_q ||x_q - x*_q||_inf / ||x_q||_inf: the size of
                            one more refinement correction relative to the solution, with the
                            factors of the rung that finished (Demmel et al., ACM TOMS 32(2),
                            2006) */
    int f32_refactor;    /* 1 if the FP32 factorization with the FP32 update was made after
                            classic refinement stalled on the tensor-core update's factors */
    int cost_stop;       /* 1 if the cost model ended the low-precision rungs early: their
                            predicted or spent refinement time reached the predicted cost of
                            the FP64 fallback */
    double t_fallback_ms;  /* host time of the FP64 fallback (factorization and refinement), 0 if none */
    double cond_est;     /* ||A||_inf ||M^{-1} r||_inf / ||r||_inf for one right-hand side r uniform in
                            [-1, 1) and M the first factorization: a lower estimate of the condition
                            number (0 when the first factorization was not made or was singular) */
} lu_mixed_report;

/*
 * lu_solve_mixed -- solve A X = B to FP64 backward error `tol` using an FP32
 * LU with a BF16 tensor-core trailing update, recovered by iterative
 * refinement with FP64 residuals; GMRES-IR and then the FP64 factorization are
 * the fallbacks when refinement stalls.  (The precision ladder is not in the
 * paper; the factorization it refines is the blocked look-ahead LU above.)
 *   dA  device FP64 n x n (lda), read only.  dB device FP64 n x nrhs (ldb),
 *   read only.  dX device FP64 n x nrhs (ldx), output.
 *   opts host pointer or NULL.  rep host pointer (may be NULL).
 *   Synchronizes `stream` before returning (to fill rep).
 *   The preconditioner solves with the FP32 factors use the inverses of their
 *   64 x 64 diagonal blocks (formed once per factorization), so a block's
 *   diagonal solve is a product rather than a chain of substitution steps.
 *   Environment: LU_MIXED_LOG=1 prints each step's backward error and time,
 *   and the cost model's prediction, to stderr.
 */
int lu_solve_mixed(int n, int nrhs, const double *dA, int lda, const double *dB, int ldb,
                   double *dX, int ldx, const lu_mixed_opts *opts, lu_mixed_report *rep,
                   void *stream);

/*
 * lu_cholesky -- A = L L^T of a symmetric positive definite n x n matrix, in
 * place (lower triangle read and overwritten; the strictly upper part is not
 * touched).  The factorization section 1 of the paper names as the next case
 * for the scheme, run on the same look-ahead schedule as lu_factor: per panel
 * of b_o <= 64 columns, the diagonal block and L21 := A21 L11^{-T} in one
 * kernel, then A22 -= L21 L21^T (lower triangle only) split into the next
 * strip (panel branch) and the rest (remainder branch).
 *   dt      LU_F64 or LU_F32.      dA, lda  as lu_factor.
 *   d_info  device int (output): 0, or j > 0 when the updated diagonal entry
 *           of column j (1-based) is not positive (the first such j; the
 *           factors past it are meaningless, as in LAPACK's potrf).
 *   opts    NULL or: nb (b_o, 1..64; 0 = 64), lookahead (-1: none), update
 *           (LU_UPDATE_NATIVE, or LU_UPDATE_F64EMU with LU_F64), spin_ns.
 */
int lu_cholesky(lu_dtype dt, int n, void *dA, int lda, int *d_info, const lu_opts *opts, void *stream);

/*
 * lu_cholesky_solve -- X := A^{-1} B with the factor of lu_cholesky: L Y = B,
 * L^T X = Y, through the substitutions of lu_solve applied to the unit lower
 * factor L diag(L)^{-1} and the upper factor diag(L) L^T (formed in a
 * stream-ordered n x n workspace).  dB device n x nrhs (ldb), overwritten.
 */
int lu_cholesky_solve(lu_dtype dt, int n, int nrhs, const void *dL, int lda, void *dB, int ldb, void *stream);

/*
 * lu_trailing_update -- the trailing update step alone (RL3 / RU2 of the
 * paper): C := C - A * B with C m x n FP32 column-major (ldc), A m x k and
 * B k x n.  `update` selects LU_UPDATE_BF16 (operands rounded to BF16,
 * tcgen05 tensor cores, FP32 accumulate), LU_UPDATE_BF16X3 (split BF16,
 * three products), LU_UPDATE_FP8 (e4m3 with power-of-two scales per row of
 * A and column of B; k <= 256) or LU_UPDATE_NATIVE (FP32 SIMT).
 * A (lda) and B (ldb) are FP32 column-major device matrices.  Exposed so
 * the update kernel can be tested and timed on its own.
 */
int lu_trailing_update(int update, int m, int n, int k, const float *dA, int lda,
                       const float *dB, int ldb, float *dC, int ldc, void *stream);

/*
 * lu_trailing_update_f64 -- the same step on FP64 matrices: C := C - A * B,
 * C m x n (ldc), A m x k (lda), B k x n (ldb), FP64 column-major device
 * matrices.  update: LU_UPDATE_NATIVE (DFMA on the CUDA cores) or
 * LU_UPDATE_F64EMU (k <= 64; A and B split into BF16 digit slices with
 * stream-ordered workspace, tcgen05 products, one FP64 rounding per element).
 */
int lu_trailing_update_f64(int update, int m, int n, int k, const double *dA, int lda,
                           const double *dB, int ldb, double *dC, int ldc, void *stream);

/*
 * Autotuner.  Section 3.1 leaves the outer panel width b_o to a trade-off (a
 * wide panel makes a fast trailing update, a narrow one a short panel chain)
 * and section 3.2 the number of threads in the panel team; here both, and the
 * batched panel width, are chosen by timing candidates on the device.
 *
 * The process-wide table maps (kind, dt, update, n) to the options that won:
 * kind 0 = lu_factor of order n (update = the LU_UPDATE_* of the call), kind 1
 * = lu_factor_batched with max_n = n (update 0).  lu_factor (and the FP32 and
 * FP64 factorizations inside lu_solve_mixed) fill every option left at zero
 * (nb, nb_inner, panel_ctas, lookahead) from the entry for their exact order;
 * lu_factor_batched with nb = 0 takes the entry's nb.  Without an entry the
 * built-in choice applies.  The table lives in host memory; calls are
 * thread-safe.
 */
typedef struct {
    lu_opts opts;     /* the fastest candidate (nb always set; other zero fields = built-in) */
    double ms;        /* its device time (best of three for n <= 4096, else one run) */
    int candidates;   /* plans timed */
} lu_tune_result;

/*
 * lu_autotune -- times lu_factor(dt, n) for candidate plans on a scratch n x n
 * matrix (entries uniform in [-1, 1), allocated stream-ordered on `stream`,
 * 2 n^2 elements) and records the fastest in the table.  Candidates: the
 * built-in plan; b_o in {16, 32, 64} (FP64), {32, 64} (emulated FP64) or
 * {64, 128, 256} (FP32 and its tensor-core updates); then panel teams of 8 and
 * 4 CTAs at the best b_o; for n <= 2048 also the plan without look-ahead; the
 * look-ahead of depth 2; for the tensor-core updates also a remainder-update
 * grid of 112 CTAs (update_ctas); for the DFMA and emulated FP64 updates both
 * tile shapes (tile 1 and 2).  budget_ms > 0 stops adding candidates once
 * that much device time has been spent (at least one is timed).
 * update: LU_UPDATE_* (BF16 .. FP8 with LU_F32, F64EMU with LU_F64).
 * Synchronizes `stream`.
 * Returns 0, a negative argument index, LU_ERR_NOMEM, LU_ERR_CUDA or
 * LU_ERR_TIMEOUT; res (host) receives the winner.
 */
int lu_autotune(lu_dtype dt, int n, int update, double budget_ms, lu_tune_result *res, void *stream);

/*
 * lu_autotune_batched -- times lu_factor_batched with nb = 16, 32 and 1 (only
 * 1 when max_n > 256) on scratch matrices of the orders in d_n (device
 * int[batch], read once), best of three runs each, and records the fastest
 * under (kind 1, dt, 0, max_n).  Synchronizes `stream`.
 */
int lu_autotune_batched(lu_dtype dt, int batch, const int *d_n, int max_n, lu_tune_result *res, void *stream);

/*
 * lu_plan_info -- the plan lu_factor(dt, n, ..., opts) would run, without any
 * CUDA call: *plan (host) receives the outer width b_o, the inner width of the
 * first panel, the panel team, lookahead (1 on, -1 off), the update kind and
 * the wait bound, after the autotuner's table and the built-in choice have
 * filled the zero fields of opts.  Returns 0 if every panel of the plan fits a
 * cluster's shared memory, LU_ERR_UNSUPPORTED if one does not (lu_factor then
 * returns the same code and launches nothing), or -i for a bad argument i.
 */
int lu_plan_info(lu_dtype dt, int n, const lu_opts *opts, lu_opts *plan);

/* Table access (host only, no CUDA calls).  lu_tune_get returns 1 and fills
 * *out when an entry exists, else 0.  lu_tune_put validates and stores an
 * entry (negative argument index on error).  lu_tune_save writes the table as
 * text (one entry per line: kind dtype update n nb nb_inner panel_ctas
 * lookahead ms; '#' starts a comment) and returns the entries written or -1;
 * lu_tune_load merges such a file and returns the entries read, -1 if it
 * cannot be read, -2 if any line is malformed or out of range (then nothing is
 * taken).  lu_tune_count returns the number of entries. */
int lu_tune_get(int kind, lu_dtype dt, int update, int n, lu_opts *out);
int lu_tune_put(int kind, lu_dtype dt, int update, int n, const lu_opts *opts, double ms);
int lu_tune_save(const char *path);
int lu_tune_load(const char *path);
int lu_tune_count(void);
void lu_tune_clear(void);

/*
 * lu_workspace_size -- bytes of internal workspace a call allocates
 * (routine: "factor", "solve", "mixed"); informational.
 */
size_t lu_workspace_size(const char *routine, int n, int nrhs, lu_dtype dt);

/* Human-readable text for a return code. */
const char *lu_status_string(int code);

/*
 * lu_last_device_status -- LU_OK or LU_ERR_TIMEOUT recorded by a bounded
 * device wait since the last reset.  Synchronizes `stream`.  reset != 0 clears
 * it afterwards.  lu_get_status(stream) is lu_last_device_status(stream, 0).
 */
int lu_last_device_status(void *stream, int reset);
int lu_get_status(void *stream);

/*
 * lu_update_timing -- instrumentation of the trailing-update launches (RL3 /
 * PF2 / RU2), used to report the update kernel against its roofline.
 *   enable != 0: from now on every trailing-update launch is bracketed by a
 *   pair of CUDA events recorded on the stream it is launched on; 0 stops.
 *   Returns 0.
 * lu_update_timing_read -- waits for the recorded events, returns the number
 *   of timed launches, their summed device time (ms), summed algorithmic
 *   flops (2 m n k per launch) and summed algorithmic bytes (C read and
 *   written once, A and B read once, at their storage widths), then clears
 *   the record.  Host pointers; any may be NULL.
 */
int lu_update_timing(int enable);
int lu_update_timing_read(long long *launches, double *total_ms, double *flops, double *bytes);

/*
 * lu_trace -- launch trace of the factorization schedule (section 4's
 * execution traces, one row per task): with enable != 0, every launch of
 * lu_factor's blocked loop is bracketed by two CUDA events on the stream it
 * runs on (stream 0: the panel stream PF, 1: the update stream RU).  Tracing
 * adds host work per launch; it is off by default.  Returns 0.
 * lu_trace_read -- waits for the recorded events and writes up to max_events
 * records into the host array out, times in ms from the earliest recorded
 * start; clears the record.  Returns the number written (with out == NULL:
 * the number recorded) or a negative status.
 */
enum {
    LU_TRACE_PANEL = 0,      /* PF3 / RL1: panel factorization of panel `step` */
    LU_TRACE_SWAP_LEFT = 1,  /* interchanges of panel `step` on the L columns to its left */
    LU_TRACE_RU1 = 2,        /* interchanges + U12 solve on the RU columns */
    LU_TRACE_PF1 = 3,        /* interchanges + U12 solve on the next panel's columns */
    LU_TRACE_PF2 = 4,        /* trailing update of the next panel's columns */
    LU_TRACE_RU2 = 5         /* trailing update of the RU columns */
};
typedef struct {
    int kind;       /* LU_TRACE_* */
    int step;       /* iteration k (for LU_TRACE_PANEL: the panel index) */
    int stream;     /* 0: PF stream, 1: RU stream */
    float t_start_ms, t_end_ms;
} lu_trace_event;
int lu_trace(int enable);
int lu_trace_read(lu_trace_event *out, int max_events);

/*
 * lu_cta_trace -- per-CTA trace of the factorization kernels, the GPU
 * counterpart of the paper's per-thread execution traces (section 4): with
 * capacity > 0, a device ring of that many records is installed and thread 0
 * of every CTA of lu_factor's panel, interchange/solve and update kernels
 * appends one record when it finishes: the task (LU_TRACE_* kind and step, as
 * in lu_trace), the CTA index, the SM it ran on, the update tiles it
 * processed (persistent update kernels; 1 per CTA for the others) and its
 * start and end in %globaltimer nanoseconds.  It shows, for instance, the SMs
 * of panel k+1's cluster picking up update tiles of step k once the panel is
 * done.  capacity 0 removes the ring.  Returns 0, LU_ERR_NOMEM or
 * LU_ERR_CUDA.  Records beyond the capacity are dropped (and counted).
 * lu_cta_trace_read -- synchronizes the device, copies up to max_events
 * records into the host array out and clears the ring; returns the number of
 * records made (which may exceed max_events or the capacity) or a negative
 * status.
 */
typedef struct {
    int kind, step;      /* LU_TRACE_* and its step */
    int cta, smid;       /* blockIdx.x and the SM (%smid) */
    int tiles;           /* update tiles taken by this CTA */
    int pad;
    unsigned long long t0_ns, t1_ns;   /* %globaltimer at start and end */
} lu_cta_event;
int lu_cta_trace(int capacity);
int lu_cta_trace_read(lu_cta_event *out, int max_events);

/*
 * lu_wait_selftest -- exercises the bounded device waits without any fault:
 * launches the blocked forward substitution on a 128 x 128 triangle with
 * the first row block withheld, so the second block's wait for it runs out
 * after bound_ns of GPU time.  Returns the status the kernel recorded
 * (LU_ERR_TIMEOUT when the bound works), synchronizing the stream; a
 * negative argument / CUDA error code otherwise.  The device stays usable.
 */
int lu_wait_selftest(long long bound_ns, void *stream);

/*
 * lu_div_selftest -- compares the substitutions' correctly rounded quotient
 * (Markstein's correction from a precomputed reciprocal) with the IEEE
 * division on `count` hashed operand pairs of type dt (seed selects them).
 * Returns the number of pairs whose results differ in any bit (0 expected),
 * synchronizing the stream; negative on an argument or CUDA error.
 */
long long lu_div_selftest(lu_dtype dt, long long count, unsigned long long seed, void *stream);

/*
 * lu_peak_probe -- measured throughput of the arithmetic units the FP64 and
 * FP32 paths run on, for roofline denominators (instrumentation; the paper
 * reports its CPU's peak the same way, as flops per cycle times the clock).
 *   kind 0: FP64 fused multiply-adds on the CUDA cores (DFMA);
 *        1: FP32 fused multiply-adds (FFMA);
 *        2: mma.sync m8n8k4 with FP64 operands (DMMA).
 *   iters: outer steps (DFMA: the compute loop of the tiled update, 16 steps
 *   of a 4 x 4 outer product per thread with operands from shared memory;
 *   FFMA: 8 independent register chains per thread; DMMA: 4 chained mma.sync
 *   per warp; 4 CTAs of 256 threads per SM).  Launches one kernel
 *   on `stream`, times it with CUDA events and synchronizes.  *tflops (host)
 *   receives flops / time / 1e12, *ms the kernel time; either may be NULL.
 *   Returns 0, -1 (bad kind), -2 (iters <= 0) or LU_ERR_CUDA.
 */
int lu_peak_probe(int kind, long long iters, double *tflops, double *ms, void *stream);

/* Number of CUDA kernels this library has launched since it was loaded. */
long long lu_kernel_launches(void);

/* Version string of the build (architecture and options). */
const char *lu_version(void);

/* sizeof of a public struct of this header, by name ("lu_opts", "lu_mixed_opts",
 * "lu_mixed_report", "lu_tune_result", "lu_trace_event", "lu_cta_event"), 0 for
 * any other name: lets a binding check its copies of these layouts against the
 * library it loaded. */
size_t lu_abi_size(const char *name);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LU_H */
