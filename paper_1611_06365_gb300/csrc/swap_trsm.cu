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
#include <cuda_bf16.h>

namespace lu {

constexpr int kSwapThreads = 256;
constexpr int kStrip = 32;          // columns per CTA
constexpr int kVS = kStrip + 1;      // row stride of the strip buffer (bank-conflict padding)
constexpr int kTrsmBlk = 32;        // diagonal block of the blocked TRSM

// map layout in global memory (written by the panel kernel): [0] = count,
// [1 .. 1+2b) rows, [1+2b .. 1+4b) src

template <typename T> __device__ __forceinline__ __nv_bfloat16 to_bf16(T v) { return __float2bfloat16_rn((float)v); }

// For the column strip [c_begin + kStrip*blockIdx.x, ... ) within [c_begin, c_end):
//   apply the row map (all rows of S), then, if do_trsm, solve
//   X := trilu(L11)^{-1} X for the b panel rows (L11 = A[kb:kb+b, kb:kb+b])
//   and store X back (and, if stage != NULL, as BF16 into stage[(c - stage_c0)*ldst + r]).
template <typename T>
__global__ void __launch_bounds__(kSwapThreads)
swap_trsm_kernel(T *__restrict__ A, int lda, int kb, int b, const int *__restrict__ map, int c_begin,
                 int c_end, int do_trsm, __nv_bfloat16 *__restrict__ stage, int ldst, int stage_c0,
                 int stage_k, int split) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cnt = map[0];
    int *rows = reinterpret_cast<int *>(smem_raw);              // [2b]
    int *src = rows + 2 * b;                                     // [2b]
    T *V = reinterpret_cast<T *>(smem_raw + (((size_t)4 * b * sizeof(int) + 15) & ~(size_t)15));
    // V: [2b][kVS], rows of S by strip column (X = first b rows)
    T *Lblk = V + (size_t)2 * b * kVS;                          // [kTrsmBlk][b] column slab of L11

    const int c0 = c_begin + blockIdx.x * kStrip;
    const int ncol = min(kStrip, c_end - c0);
    if (ncol <= 0) return;
    for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
        rows[s] = map[1 + s];
        src[s] = map[1 + 2 * b + s];
    }
    __syncthreads();
    // gather old values (threads run down S for a fixed column: coalesced for the panel rows)
    for (int e = threadIdx.x; e < cnt * ncol; e += blockDim.x) {
        const int s = e % cnt, c = e / cnt;
        V[(size_t)s * kVS + c] = A[(size_t)src[s] + (size_t)(c0 + c) * lda];
    }
    __syncthreads();
    // scatter rows outside the panel (and, without a solve, the panel rows too)
    const int first = do_trsm ? b : 0;
    for (int e = threadIdx.x; e < (cnt - first) * ncol; e += blockDim.x) {
        const int s = first + e % (cnt - first), c = e / (cnt - first);
        A[(size_t)rows[s] + (size_t)(c0 + c) * lda] = V[(size_t)s * kVS + c];
    }
    if (!do_trsm) return;

    // blocked forward substitution with unit lower L11 on X = V[0:b][0:ncol]
    const int tc = threadIdx.x % kStrip, tg = threadIdx.x / kStrip, ng = kSwapThreads / kStrip;
    for (int d0 = 0; d0 < b; d0 += kTrsmBlk) {
        const int db = min(kTrsmBlk, b - d0);
        // stage the column slab L11[d0:b, d0:d0+db] (rows d0..b-1)
        __syncthreads();
        const int slab_rows = b - d0;
        for (int e = threadIdx.x; e < slab_rows * db; e += blockDim.x) {
            const int r = e % slab_rows, c = e / slab_rows;
            Lblk[(size_t)c * b + r] = A[(size_t)(kb + d0 + r) + (size_t)(kb + d0 + c) * lda];
        }
        // diagonal block: rows in parallel, one step per column of L
        for (int jj = 0; jj < db; ++jj) {
            __syncthreads();
            if (tc < ncol) {
                const T x = V[(size_t)(d0 + jj) * kVS + tc];
                for (int ii = jj + 1 + tg; ii < db; ii += ng)
                    V[(size_t)(d0 + ii) * kVS + tc] = fma(-Lblk[(size_t)jj * b + ii], x, V[(size_t)(d0 + ii) * kVS + tc]);
            }
        }
        __syncthreads();
        // rows below the diagonal block: X[r] -= L[r, d0:d0+db] X[d0:d0+db]
        const int below = b - d0 - db;
        for (int e = threadIdx.x; e < below * ncol; e += blockDim.x) {
            const int c = e % ncol, r = e / ncol;
            T acc = V[(size_t)(d0 + db + r) * kVS + c];
            for (int jj = 0; jj < db; ++jj)
                acc = fma(-Lblk[(size_t)jj * b + db + r], V[(size_t)(d0 + jj) * kVS + c], acc);
            V[(size_t)(d0 + db + r) * kVS + c] = acc;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * ncol; e += blockDim.x) {
        const int r = e % b, c = e / b;
        const T x = V[(size_t)r * kVS + c];
        A[(size_t)(kb + r) + (size_t)(c0 + c) * lda] = x;
        if (stage) {
            const __nv_bfloat16 hi = to_bf16(x);
            stage[(size_t)(c0 + c - stage_c0) * ldst + r] = hi;
            if (split) stage[(size_t)(c0 + c - stage_c0) * ldst + stage_k + r] = to_bf16((float)x - __bfloat162float(hi));
        }
    }
    if (stage) {   // zero K padding (b < stage_k on a short last panel)
        for (int e = threadIdx.x; e < (stage_k - b) * ncol; e += blockDim.x) {
            const int r = b + e % (stage_k - b), c = e / (stage_k - b);
            stage[(size_t)(c0 + c - stage_c0) * ldst + r] = __float2bfloat16_rn(0.f);
            if (split) stage[(size_t)(c0 + c - stage_c0) * ldst + stage_k + r] = __float2bfloat16_rn(0.f);
        }
    }
}

size_t swap_trsm_smem_bytes(int b, size_t elem) {
    size_t a = (size_t)4 * b * sizeof(int);
    a = (a + 15) & ~(size_t)15;
    a += (size_t)2 * b * kVS * elem;
    a += (size_t)kTrsmBlk * b * elem;
    return a + 16;
}

template <typename T>
cudaError_t launch_swap_trsm(T *A, int lda, int kb, int b, const int *map, int c_begin, int c_end,
                             int do_trsm, __nv_bfloat16 *stage, int ldst, int stage_c0, int stage_k, int split,
                             cudaStream_t s) {
    if (c_end <= c_begin) return cudaSuccess;
    size_t smem = swap_trsm_smem_bytes(b, sizeof(T));
    static bool attr_set[2] = {false, false};
    if (!attr_set[sizeof(T) == 8]) {
        cudaError_t e = cudaFuncSetAttribute(swap_trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[sizeof(T) == 8] = true;
    }
    int grid = lu_ceil_div(c_end - c_begin, kStrip);
    swap_trsm_kernel<T><<<grid, kSwapThreads, smem, s>>>(A, lda, kb, b, map, c_begin, c_end, do_trsm,
                                                         stage, ldst, stage_c0, stage_k, split);
    return cudaGetLastError();
}

template cudaError_t launch_swap_trsm<double>(double *, int, int, int, const int *, int, int, int, __nv_bfloat16 *, int, int, int, int, cudaStream_t);
template cudaError_t launch_swap_trsm<float>(float *, int, int, int, const int *, int, int, int, __nv_bfloat16 *, int, int, int, int, cudaStream_t);

}  // namespace lu
