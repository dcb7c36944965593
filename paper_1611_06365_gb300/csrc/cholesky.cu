// Cholesky factorization A = L L^T (lower) of a symmetric positive definite
// matrix, on the same look-ahead schedule as the LU factorization: the
// factorization section 1 of the paper names as the next case for the
// scheme (the panel, its solve and the trailing update are the three tasks;
// there is no pivoting, so no interchanges and no row maps).
//
// Blocked right-looking, panel width b_o <= 64.  Per step k:
//   panel(k)  the w x w diagonal block is factored in shared memory, l_jj =
//             sqrt of the updated diagonal, l_ij = a_ij / l_jj, rank-1 update
//             of the block's lower triangle (every CTA factors it, so no CTA
//             waits for another), then every thread solves one row of
//             L21 := A21 L11^{-T} in registers (forward substitution in
//             increasing column order, as the unblocked elimination updates
//             each element) and stages it for the emulated FP64 update;
//   PF2(k)    A22 -= L21 L21^T on the next strip of b_o columns (panel branch);
//   RU2(k)    the same on the columns right of it, lower triangle only
//             (remainder branch).
// The update is the DFMA tile kernel with B read transposed, or the emulated
// FP64 tensor-core kernel with B's digit slices taken from the same staged
// rows as A; both write only the lower triangle.  Two streams ordered by
// events, as for the LU factorization (section 3.2, Figure 3).
#include "common.cuh"
#include "internal.h"
#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

namespace lu {

constexpr int kChW = 64;          // widest panel
constexpr int kChThreads = 256;   // one row of L21 per thread

template <typename T>
__global__ void __launch_bounds__(kChThreads)
chol_panel(T *__restrict__ A, int lda, int m, int w, int kb_abs, int *__restrict__ info, int *__restrict__ arrive,
           StageDesc sd, CtaTrace tr) {
    const unsigned long long t_start = tr.ring ? lu_globaltimer() : 0ull;
    __shared__ T D[kChW][kChW + 1];
    __shared__ int bad, last;
    const int tid = threadIdx.x;
    if (tid == 0) bad = -1;
    for (int e = tid; e < w * w; e += kChThreads) {
        const int r = e % w, c = e / w;
        D[r][c] = r >= c ? A[(size_t)r + (size_t)c * lda] : T(0);
    }
    __syncthreads();
    // the last CTA to have read the diagonal block writes its factor back (every CTA
    // computes the same one); it resets the counter for the next panel
    if (tid == 0) {
        __threadfence();
        const int old = atomicAdd(arrive, 1);
        last = old == (int)gridDim.x - 1;
        if (last) atomicExch(arrive, 0);
    }
    // the diagonal block, column by column (identical in every CTA)
    for (int j = 0; j < w; ++j) {
        const T d = D[j][j];
        if (!(d > T(0)) && tid == 0 && bad < 0) bad = j;
        const T l = sqrt(d);
        __syncthreads();   // every thread has read D[j][j]
        if (tid == 0) D[j][j] = l;
        for (int i = j + 1 + tid; i < w; i += kChThreads) D[i][j] = D[i][j] / l;
        __syncthreads();
        const int r = w - j - 1;
        for (int e = tid; e < r * r; e += kChThreads) {
            const int i = j + 1 + e % r, c = j + 1 + e / r;
            if (i >= c) D[i][c] = fma(-D[i][j], D[c][j], D[i][c]);
        }
        __syncthreads();
    }
    if (last) {
        if (tid == 0 && bad >= 0) atomicCAS(info, 0, kb_abs + bad + 1);
        for (int e = tid; e < w * w; e += kChThreads) {
            const int r = e % w, c = e / w;
            if (r >= c) A[(size_t)r + (size_t)c * lda] = D[r][c];
        }
    }
    // one row of L21 per thread: x L11^T = a, columns in increasing order
    const int i = w + (int)blockIdx.x * kChThreads + tid;
    if (i < m) {
        T x[kChW];
#pragma unroll
        for (int c = 0; c < kChW; ++c) x[c] = c < w ? A[(size_t)i + (size_t)c * lda] : T(0);
#pragma unroll
        for (int k = 0; k < kChW; ++k) {
            if (k < w) {
                x[k] = x[k] / D[k][k];
#pragma unroll
                for (int c = k + 1; c < kChW; ++c)
                    if (c < w) x[c] = fma(-x[k], D[c][k], x[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < kChW; ++c)
            if (c < w) A[(size_t)i + (size_t)c * lda] = x[c];
        if constexpr (sizeof(T) == 8) {
            if (sd.ptr && sd.fmt == 3) {
                // digit slices of the row for the emulated FP64 update (stage row i - w)
                unsigned long long amax = 0;
#pragma unroll
                for (int c = 0; c < kChW; ++c) amax = max(amax, c < w ? lu_f64_abs_bits(x[c]) : 0ull);
                const int ex = lu_f64_scale_exp_bits(amax);
                sd.dscale[i - w] = ldexp(1.0, ex);
                __nv_bfloat16 *dst = static_cast<__nv_bfloat16 *>(sd.ptr) + (size_t)(i - w) * sd.lds;
                // the row just stored, read back (cached) so the slicing is not unrolled over the tile
#pragma unroll 1
                for (int c = 0; c < sd.kpad; ++c)
                    lu_f64_slices(c < w ? (double)A[(size_t)i + (size_t)c * lda] : 0.0, ex, dst + c, (size_t)sd.kpad);
            }
        }
    }
    if (tid == 0) lu_trace_cta(tr, t_start, 0);
}

template <typename T>
cudaError_t launch_chol_panel(T *A, int lda, int m, int w, int kb_abs, int *info, int *arrive, StageDesc sd, cudaStream_t s,
                              CtaTrace tr) {
    if (m <= 0 || w <= 0) return cudaSuccess;
    if (w > kChW) return cudaErrorInvalidValue;
    const int grid = std::max(1, lu_ceil_div(m - w, kChThreads));
    chol_panel<T><<<grid, kChThreads, 0, s>>>(A, lda, m, w, kb_abs, info, arrive, sd, tr);
    lu_count_launch();
    return cudaGetLastError();
}

// The factors of A = L L^T in the form lu_solve takes (no interchanges):
// A = Lh (D L^T) with Lh = L D^{-1} unit lower and D = diag(L), so W(i, j) =
// L(i, j) / L(j, j) below the diagonal and W(i, j) = L(i, i) L(j, i) on and
// above it.
template <typename T>
__global__ void chol_to_lu(int n, const T *__restrict__ L, int ldl, T *__restrict__ W, int ldw) {
    const size_t total = (size_t)n * n;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        T v;
        if (i > j) v = L[(size_t)i + (size_t)j * ldl] / L[(size_t)j + (size_t)j * ldl];
        else v = L[(size_t)i + (size_t)i * ldl] * L[(size_t)j + (size_t)i * ldl];   // U(i, j) = L(i, i) L(j, i)
        W[(size_t)i + (size_t)j * ldw] = v;
    }
}

}  // namespace lu

using namespace lu;

namespace {

constexpr int kChMaxDev = 64;

struct ChDev {
    bool init = false;
    cudaStream_t P = nullptr, U = nullptr;
    cudaEvent_t evIn = nullptr, evP[2] = {}, evU[2] = {}, evPF2 = nullptr, evOutP = nullptr, evOutU = nullptr;
};
ChDev g_ch[kChMaxDev];
std::mutex g_ch_mu;

cudaError_t ch_dev(ChDev **out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kChMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_ch_mu);
    ChDev &st = g_ch[d];
    if (!st.init) {
        int lo = 0, hi = 0;
        if ((e = cudaDeviceGetStreamPriorityRange(&lo, &hi)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithPriority(&st.P, cudaStreamNonBlocking, hi)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithPriority(&st.U, cudaStreamNonBlocking, lo)) != cudaSuccess) return e;
        cudaEvent_t *evs[] = {&st.evIn, &st.evP[0], &st.evP[1], &st.evU[0], &st.evU[1], &st.evPF2, &st.evOutP, &st.evOutU};
        for (cudaEvent_t *ev : evs)
            if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess) return e;
        st.init = true;
    }
    *out = &st;
    return cudaSuccess;
}

struct ChWork {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit ChWork(cudaStream_t st) : s(st) {}
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        void *v = nullptr;
        cudaError_t e = cudaMallocAsync(&v, std::max<size_t>(count, 1) * sizeof(T), s);
        if (e != cudaSuccess) return e;
        ptrs.push_back(v);
        *p = static_cast<T *>(v);
        return cudaSuccess;
    }
    ~ChWork() {
        for (void *v : ptrs) cudaFreeAsync(v, s);
    }
};

template <typename T>
struct ChCtx {
    int n, lda, bo;
    T *A;
    bool emu = false;
    __nv_bfloat16 *st[2] = {nullptr, nullptr};   // digit slices of L21 per panel parity
    double *sc[2] = {nullptr, nullptr};
    CUtensorMap mapA[2], mapB[2];
    int *ctr = nullptr;      // [0], [1]: tile queues of the two branches; [2]: panel arrival counter
    int kinner = 0;
    long long bound = 0;
};

// A22 rows/cols [c0, ...) restricted to columns [c0, c1): -= L21(rows c0.., panel k) L21(rows c0..c1, panel k)^T
template <typename T>
cudaError_t chol_update(ChCtx<T> &c, int par, int kb, int w, int c0, int c1, int ctr_slot, cudaStream_t s, CtaTrace tr) {
    const int r0 = kb + w;            // first row of L21
    const int m = c.n - c0, nn = c1 - c0;
    if (m <= 0 || nn <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 8) {
        if (c.emu)
            return launch_gemm_f64emu(m, nn, c.mapA[par], c0 - r0, c.mapB[par], c0 - r0,
                                      reinterpret_cast<double *>(c.A) + c0 + (size_t)c0 * c.lda, c.lda, c.sc[par], c.sc[par],
                                      c.ctr + ctr_slot, lu_device_status_ptr(), c.bound, 0, s, tr, 0, SmShare{}, 0);
    }
    const T *L21 = c.A + c0 + (size_t)kb * c.lda;
    return launch_gemm_simt<T>(m, nn, w, L21, c.lda, L21, c.lda, c.A + c0 + (size_t)c0 * c.lda, c.lda, s, tr, true, 0, 0);
}

template <typename T>
int chol_core(int n, T *A, int lda, int *info, int bo, bool lookahead, bool emu, long long bound, cudaStream_t caller) {
    ChDev *st = nullptr;
    LU_CUDA_TRY(ch_dev(&st));
    LU_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), caller));
    if (n == 0) return LU_OK;
    ChWork ws(caller);
    ChCtx<T> c;
    c.n = n; c.lda = lda; c.bo = bo; c.A = A; c.emu = emu; c.bound = bound;
    LU_CUDA_TRY(ws.get(&c.ctr, 3));
    LU_CUDA_TRY(cudaMemsetAsync(c.ctr + 2, 0, sizeof(int), caller));
    if (emu) {
        c.kinner = f64emu_kpad() * kF64Slices;
        for (int i = 0; i < 2; ++i) {
            LU_CUDA_TRY(ws.get(&c.st[i], (size_t)n * c.kinner));
            LU_CUDA_TRY(ws.get(&c.sc[i], (size_t)n));
            LU_CUDA_TRY(make_stage_map(&c.mapA[i], c.st[i], c.kinner, n, c.kinner, f64emu_box_rows(), 0));
            LU_CUDA_TRY(make_stage_map(&c.mapB[i], c.st[i], c.kinner, n, c.kinner, f64emu_box_cols(), 0));
        }
    }
    cudaStream_t P = st->P, U = st->U;
    LU_CUDA_TRY(cudaEventRecord(st->evIn, caller));
    LU_CUDA_TRY(cudaStreamWaitEvent(P, st->evIn, 0));
    LU_CUDA_TRY(cudaStreamWaitEvent(U, st->evIn, 0));
    auto panel = [&](int kb, int w, int par, cudaStream_t s, int step) {
        StageDesc sd{nullptr, nullptr, c.kinner, emu ? f64emu_kpad() : 0, emu ? 3 : 0, nullptr};
        if (emu && kb + w < n) { sd.ptr = c.st[par]; sd.dscale = c.sc[par]; }
        return launch_chol_panel<T>(A + kb + (size_t)kb * lda, lda, n - kb, w, kb, info, c.ctr + 2, sd, s,
                                    cta_tag_ext(LU_TRACE_PANEL, step));
    };
    const int nblk = (n + bo - 1) / bo;
    LU_CUDA_TRY(panel(0, std::min(bo, n), 0, P, 0));
    LU_CUDA_TRY(cudaEventRecord(st->evP[0], P));
    for (int k = 0; k < nblk; ++k) {
        const int kb = k * bo, w = std::min(bo, n - kb), par = k & 1;
        const int cn0 = kb + w, wn = std::min(bo, n - cn0);
        const int rest0 = lookahead ? cn0 + wn : cn0;
        LU_CUDA_TRY(cudaStreamWaitEvent(U, st->evP[par], 0));
        if (wn > 0 && lookahead) {
            if (k > 0) LU_CUDA_TRY(cudaStreamWaitEvent(P, st->evU[par ^ 1], 0));
            LU_CUDA_TRY(chol_update<T>(c, par, kb, w, cn0, cn0 + wn, 0, P, cta_tag_ext(LU_TRACE_PF2, k)));
            LU_CUDA_TRY(cudaEventRecord(st->evPF2, P));
            LU_CUDA_TRY(panel(cn0, wn, par ^ 1, P, k + 1));
            LU_CUDA_TRY(cudaEventRecord(st->evP[par ^ 1], P));
            LU_CUDA_TRY(cudaStreamWaitEvent(U, st->evPF2, 0));
        }
        if (rest0 < n) LU_CUDA_TRY(chol_update<T>(c, par, kb, w, rest0, n, 1, U, cta_tag_ext(LU_TRACE_RU2, k)));
        LU_CUDA_TRY(cudaEventRecord(st->evU[par], U));
        if (wn > 0 && !lookahead) {
            LU_CUDA_TRY(cudaStreamWaitEvent(P, st->evU[par], 0));
            LU_CUDA_TRY(panel(cn0, wn, par ^ 1, P, k + 1));
            LU_CUDA_TRY(cudaEventRecord(st->evP[par ^ 1], P));
        }
    }
    LU_CUDA_TRY(cudaEventRecord(st->evOutP, P));
    LU_CUDA_TRY(cudaEventRecord(st->evOutU, U));
    LU_CUDA_TRY(cudaStreamWaitEvent(caller, st->evOutP, 0));
    LU_CUDA_TRY(cudaStreamWaitEvent(caller, st->evOutU, 0));
    LU_CUDA_TRY(cudaGetLastError());
    return LU_OK;
}

}  // namespace

extern "C" int lu_cholesky(lu_dtype dt, int n, void *dA, int lda, int *d_info, const lu_opts *opts, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (n < 0) return -2;
    if (n > 0 && !dA) return -3;
    if (lda < std::max(1, n)) return -4;
    if (!d_info) return -5;
    if (opts && (opts->nb < 0 || opts->nb > kChW ||
                 (opts->update != LU_UPDATE_NATIVE && !(opts->update == LU_UPDATE_F64EMU && dt == LU_F64))))
        return -6;
    const int bo = (opts && opts->nb > 0) ? opts->nb : kChW;
    const bool lookahead = !(opts && opts->lookahead < 0);
    const bool emu = opts && opts->update == LU_UPDATE_F64EMU;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long bound = lu_spin_bound_ns(opts);
    if (dt == LU_F64) return chol_core<double>(n, static_cast<double *>(dA), lda, d_info, bo, lookahead, emu, bound, s);
    return chol_core<float>(n, static_cast<float *>(dA), lda, d_info, bo, lookahead, false, bound, s);
}

extern "C" int lu_cholesky_solve(lu_dtype dt, int n, int nrhs, const void *dL, int lda, void *dB, int ldb, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (n > 0 && !dL) return -4;
    if (lda < std::max(1, n)) return -5;
    if (n > 0 && nrhs > 0 && !dB) return -6;
    if (ldb < std::max(1, n)) return -7;
    if (n == 0 || nrhs == 0) return LU_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ChWork ws(s);
    int *perm = nullptr;
    LU_CUDA_TRY(ws.get(&perm, n));
    LU_CUDA_TRY(launch_iota(perm, n, s));
    const size_t total = (size_t)n * n;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    if (dt == LU_F64) {
        double *W = nullptr;
        LU_CUDA_TRY(ws.get(&W, total));
        chol_to_lu<double><<<grid, 256, 0, s>>>(n, static_cast<const double *>(dL), lda, W, n);
        lu_count_launch();
        LU_CUDA_TRY(cudaGetLastError());
        return solve_f64_perm(n, nrhs, W, n, perm, static_cast<double *>(dB), ldb, s);
    }
    float *W = nullptr;
    LU_CUDA_TRY(ws.get(&W, total));
    chol_to_lu<float><<<grid, 256, 0, s>>>(n, static_cast<const float *>(dL), lda, W, n);
    lu_count_launch();
    LU_CUDA_TRY(cudaGetLastError());
    return solve_f32_perm(n, nrhs, W, n, perm, static_cast<float *>(dB), ldb, s);
}
