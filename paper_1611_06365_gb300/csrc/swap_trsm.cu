// Row interchanges outside the panel (LAPACK laswp) fused with the triangular
// solve RL2 / PF1 / RU1: A12 := trilu(A11)^{-1} A12 (section 3.1, Figure 1
// right; section 3.2, Figure 3).
//
// The b interchanges of a panel are first turned into one row map (built at
// the end of the panel kernel): the set S of rows they touch (the b panel rows
// plus every distinct target row) and, for each row of S, the row whose old
// content it receives.  Applying the interchanges in order equals one gather/scatter over
// S, so every column strip can then be processed independently and in
// parallel -- the paper notes the permutation is embarrassingly parallel
// (section 3.1) and spreads it over all threads (section 3.2).
#include "common.cuh"
#include "internal.h"
#include <cuda_bf16.h>

namespace lu {

constexpr int kSwapThreads = 256;
constexpr int kStrip = 32;          // columns per CTA
constexpr int kVS = kStrip + 1;      // row stride of the strip buffer (bank-conflict padding)
constexpr int kBelowRows = 64;      // rows of L staged per pass of the off-diagonal update

// Diagonal block of the blocked solve: 32 rows, one per lane.
template <typename T> struct TrsmBlk { static constexpr int value = 32; };

// map layout in global memory (written by the panel kernel): [0] = count,
// [1 .. 1+2b) rows, [1+2b .. 1+4b) src

template <typename T> __device__ __forceinline__ __nv_bfloat16 to_bf16(T v) { return __float2bfloat16_rn((float)v); }

// Shared memory: rows/src [4b ints] | V [2b][kVS] | Ld [DB][DB + 1] (row-major) | Lc [kBelowRows][DB + 4]
template <typename T>
struct SwapLayout {
    size_t v_off, ld_off, lc_off, total;
    __host__ __device__ explicit SwapLayout(int b) {
        constexpr int DB = TrsmBlk<T>::value;
        v_off = (((size_t)4 * b * sizeof(int)) + 15) & ~(size_t)15;
        ld_off = v_off + ((((size_t)2 * b * kVS * sizeof(T)) + 15) & ~(size_t)15);
        lc_off = ld_off + (((size_t)DB * (DB + 1) * sizeof(T) + 15) & ~(size_t)15);
        total = lc_off + (size_t)kBelowRows * (DB + 4) * sizeof(T) + 16;
    }
};

// For the column strip [c_begin + kStrip*blockIdx.x, ... ) within [c_begin, c_end):
//   apply the row map (all rows of S), then, if do_trsm, solve
//   X := trilu(L11)^{-1} X for the b panel rows (L11 = A[kb:kb+b, kb:kb+b])
//   and store X back (and, if sd.ptr != NULL, staged for the tensor-core update
//   as column c - stage_c0 of the staging buffer: BF16, BF16 hi/lo or FP8 with
//   a power-of-two scale per column).
// The solve is blocked by DB = 32 rows.  In a diagonal block lane r of every
// warp holds row r of L and of the warp's strip columns in registers; step k
// broadcasts the finished x[k] with a shuffle and lanes r > k subtract
// L[r][k] x[k] (every element takes its updates in increasing k, as in the
// unblocked substitution).  Then all threads update the rows below,
// X[r] -= L[r, blk] X[blk].
template <typename T>
__global__ void __launch_bounds__(kSwapThreads, 2)
swap_trsm_kernel(T *__restrict__ A, int lda, int kb, int b, const int *__restrict__ map, int c_begin,
                 int c_end, int do_trsm, StageDesc sd, int stage_c0, CtaTrace tr) {
    const unsigned long long t_start = tr.ring ? lu_globaltimer() : 0ull;
    constexpr int DB = TrsmBlk<T>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SwapLayout<T> lay(b);
    const int cnt = map[0];
    int *rows = reinterpret_cast<int *>(smem_raw);              // [2b]
    int *src = rows + 2 * b;                                     // [2b]
    T *V = reinterpret_cast<T *>(smem_raw + lay.v_off);          // [2b][kVS], rows of S by strip column (X = first b rows)
    T *Ld = reinterpret_cast<T *>(smem_raw + lay.ld_off);        // [DB][DB + 1] diagonal block of L11, row-major
    T *Lc = reinterpret_cast<T *>(smem_raw + lay.lc_off);        // [kBelowRows][DB + 4] rows of L below the block

    const int c0 = c_begin + blockIdx.x * kStrip;
    const int ncol = min(kStrip, c_end - c0);
    if (ncol <= 0) return;
    const int tid = threadIdx.x;
    for (int s = tid; s < cnt; s += blockDim.x) {
        rows[s] = map[1 + s];
        src[s] = map[1 + 2 * b + s];
    }
    __syncthreads();
    // gather old values (threads run down S for a fixed column: coalesced for the panel rows)
    for (int e = tid; e < cnt * ncol; e += blockDim.x) {
        const int s = e % cnt, c = e / cnt;
        V[(size_t)s * kVS + c] = A[(size_t)src[s] + (size_t)(c0 + c) * lda];
    }
    __syncthreads();
    // scatter rows outside the panel (and, without a solve, the panel rows too)
    const int first = do_trsm ? b : 0;
    for (int e = tid; e < (cnt - first) * ncol; e += blockDim.x) {
        const int s = first + e % (cnt - first), c = e / (cnt - first);
        A[(size_t)rows[s] + (size_t)(c0 + c) * lda] = V[(size_t)s * kVS + c];
    }
    if (!do_trsm) {
        if (tid == 0) lu_trace_cta(tr, t_start, 1);
        return;
    }

    const T *L11 = A + (size_t)kb + (size_t)kb * lda;
    for (int d0 = 0; d0 < b; d0 += DB) {
        const int db = min(DB, b - d0);
        // diagonal block (strictly lower part; zero outside the block), row-major
        for (int e = tid; e < DB * DB; e += blockDim.x) {
            const int r = e % DB, k = e / DB;
            Ld[(size_t)r * (DB + 1) + k] = (r > k && r < db && k < db) ? L11[(size_t)(d0 + r) + (size_t)(d0 + k) * lda] : T(0);
        }
        __syncthreads();
        {
            constexpr int CPW = kStrip / (kSwapThreads / 32);   // strip columns per warp
            const int r = tid & 31, cw = (tid >> 5) * CPW;
            T lrow[DB];
#pragma unroll
            for (int k = 0; k < DB; ++k) lrow[k] = Ld[(size_t)r * (DB + 1) + k];
            T x[CPW];
#pragma unroll
            for (int u = 0; u < CPW; ++u) x[u] = (r < db && cw + u < ncol) ? V[(size_t)(d0 + r) * kVS + cw + u] : T(0);
#pragma unroll
            for (int k = 0; k < DB - 1; ++k) {
#pragma unroll
                for (int u = 0; u < CPW; ++u) {
                    const T xk = __shfl_sync(0xffffffffu, x[u], k);
                    if (r > k) x[u] = fma(-lrow[k], xk, x[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < CPW; ++u)
                if (r < db && cw + u < ncol) V[(size_t)(d0 + r) * kVS + cw + u] = x[u];
        }
        __syncthreads();
        // rows below the block: X[r] -= L[r, d0:d0+db] X[d0:d0+db], kBelowRows rows per pass
        for (int rb = d0 + db; rb < b; rb += kBelowRows) {
            const int nr = min(kBelowRows, b - rb);
            for (int e = tid; e < kBelowRows * DB; e += blockDim.x) {
                const int r = e % kBelowRows, k = e / kBelowRows;
                Lc[(size_t)r * (DB + 4) + k] = (r < nr && k < db) ? L11[(size_t)(rb + r) + (size_t)(d0 + k) * lda] : T(0);
            }
            __syncthreads();
            {
                // thread: column c, rows rq + 8 i (i < 8); each element takes its
                // updates in increasing k, as in the unblocked substitution
                const int c = tid & 31, rq = tid >> 5;
                T acc[kBelowRows / 8];
#pragma unroll
                for (int i = 0; i < kBelowRows / 8; ++i) {
                    const int r = rq + 8 * i;
                    acc[i] = (r < nr && c < ncol) ? V[(size_t)(rb + r) * kVS + c] : T(0);
                }
                for (int k = 0; k < db; k += 4) {
                    T xv[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) xv[v] = (k + v < db) ? V[(size_t)(d0 + k + v) * kVS + c] : T(0);
#pragma unroll
                    for (int i = 0; i < kBelowRows / 8; ++i) {
                        const T *lr = Lc + (size_t)(rq + 8 * i) * (DB + 4) + k;
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[i] = fma(-lr[v], xv[v], acc[i]);
                    }
                }
                if (c < ncol) {
#pragma unroll
                    for (int i = 0; i < kBelowRows / 8; ++i) {
                        const int r = rq + 8 * i;
                        if (r < nr) V[(size_t)(rb + r) * kVS + c] = acc[i];
                    }
                }
            }
            __syncthreads();
        }
    }
    if (sd.ptr && sd.fmt == 2) {
        // FP8 staging: one power-of-two scale per column, 8 threads per column
        float *colmul = reinterpret_cast<float *>(Lc);
        const int c = tid >> 3, sub = tid & 7;
        float amax = 0.f;
        if (c < ncol)
            for (int r = sub; r < b; r += 8) amax = fmaxf(amax, fabsf((float)V[(size_t)r * kVS + c]));
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        float inv;
        const float mul = lu_fp8_scale(amax, &inv);
        if (sub == 0 && c < ncol) {
            colmul[c] = mul;
            sd.scale[c0 + c - stage_c0] = inv;
        }
        __syncthreads();
    }
    if (sd.ptr && sd.fmt == 3) {
        // FP64 digit slices: one power-of-two scale per column, 8 threads per column
        int *colexp = reinterpret_cast<int *>(Lc);
        const int c = tid >> 3, sub = tid & 7;
        unsigned long long amax = 0;
        if (c < ncol)
            for (int r = sub; r < b; r += 8) amax = max(amax, lu_f64_abs_bits((double)V[(size_t)r * kVS + c]));
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        if (sub == 0 && c < ncol) {
            const int ex = lu_f64_scale_exp_bits(amax);
            colexp[c] = ex;
            sd.dscale[c0 + c - stage_c0] = ldexp(1.0, ex);
        }
        __syncthreads();
        __nv_bfloat16 *st16 = static_cast<__nv_bfloat16 *>(sd.ptr);
        for (int e = tid; e < sd.kpad * ncol; e += blockDim.x) {
            const int r = e % sd.kpad, cc = e / sd.kpad;
            const double x = r < b ? (double)V[(size_t)r * kVS + cc] : 0.0;
            lu_f64_slices(x, colexp[cc], st16 + (size_t)(c0 + cc - stage_c0) * sd.lds + r, (size_t)sd.kpad);
        }
        for (int e = tid; e < b * ncol; e += blockDim.x) {
            const int r = e % b, cc = e / b;
            A[(size_t)(kb + r) + (size_t)(c0 + cc) * lda] = V[(size_t)r * kVS + cc];
        }
        if (tid == 0) lu_trace_cta(tr, t_start, 1);
        return;
    }
    const int kpad = sd.kpad;
    for (int e = tid; e < b * ncol; e += blockDim.x) {
        const int r = e % b, c = e / b;
        const T x = V[(size_t)r * kVS + c];
        A[(size_t)(kb + r) + (size_t)(c0 + c) * lda] = x;
        if (sd.ptr) {
            const size_t col = (size_t)(c0 + c - stage_c0) * sd.lds;
            if (sd.fmt == 2) {
                static_cast<unsigned char *>(sd.ptr)[col + r] = lu_to_e4m3((float)x * reinterpret_cast<const float *>(Lc)[c]);
            } else {
                __nv_bfloat16 *st16 = static_cast<__nv_bfloat16 *>(sd.ptr);
                const __nv_bfloat16 hi = to_bf16(x);
                st16[col + r] = hi;
                if (sd.fmt == 1) st16[col + kpad + r] = to_bf16((float)x - __bfloat162float(hi));
            }
        }
    }
    if (sd.ptr) {   // zero K padding (b < kpad on a short last panel)
        for (int e = tid; e < (kpad - b) * ncol; e += blockDim.x) {
            const int r = b + e % (kpad - b), c = e / (kpad - b);
            const size_t col = (size_t)(c0 + c - stage_c0) * sd.lds;
            if (sd.fmt == 2) {
                static_cast<unsigned char *>(sd.ptr)[col + r] = 0;
            } else {
                __nv_bfloat16 *st16 = static_cast<__nv_bfloat16 *>(sd.ptr);
                st16[col + r] = __float2bfloat16_rn(0.f);
                if (sd.fmt == 1) st16[col + kpad + r] = __float2bfloat16_rn(0.f);
            }
        }
    }
    if (tid == 0) lu_trace_cta(tr, t_start, 1);
}

size_t swap_trsm_smem_bytes(int b, size_t elem) {
    return elem == 8 ? SwapLayout<double>(b).total : SwapLayout<float>(b).total;
}

template <typename T>
cudaError_t launch_swap_trsm(T *A, int lda, int kb, int b, const int *map, int c_begin, int c_end,
                             int do_trsm, StageDesc sd, int stage_c0, cudaStream_t s, CtaTrace tr) {
    if (c_end <= c_begin) return cudaSuccess;
    size_t smem = swap_trsm_smem_bytes(b, sizeof(T));
    // set on every launch: the attribute belongs to the current device's context
    cudaError_t e = cudaFuncSetAttribute(swap_trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    int grid = lu_ceil_div(c_end - c_begin, kStrip);
    swap_trsm_kernel<T><<<grid, kSwapThreads, smem, s>>>(A, lda, kb, b, map, c_begin, c_end, do_trsm, sd, stage_c0, tr);
    return cudaGetLastError();
}

template cudaError_t launch_swap_trsm<double>(double *, int, int, int, const int *, int, int, int, StageDesc, int, cudaStream_t,
                                              CtaTrace);
template cudaError_t launch_swap_trsm<float>(float *, int, int, int, const int *, int, int, int, StageDesc, int, cudaStream_t,
                                             CtaTrace);

}  // namespace lu
