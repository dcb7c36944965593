// Trailing update RL3 / PF2 / RU2 on CUDA cores: C := C - A * B
// (section 3.1, Figure 1 right; section 3.2, Figure 3).
//
// FP64 on GB300 runs at the same rate on DFMA and on the legacy DMMA path
// (about 1 TFLOP/s for the whole GPU), and the update's arithmetic intensity
// (2b/16 flop/byte for b >= 8) is far above the FP64 machine balance, so a
// register-tiled DFMA kernel is bound by the FP64 pipe, not by memory.  The
// same kernel in FP32 serves the FP32-native factorization.
//
// Tile TM x TN per CTA, 4 x 4 outputs per thread, K staged through shared
// memory in chunks of 16: 64 x 64 (256 threads) when the update has at least
// one tile per SM, else 32 x 32 (64 threads) so that a narrow update (the
// look-ahead strip of a small matrix) spreads over four times as many SMs.
// Every element accumulates its k products in increasing k and is then
// subtracted from C, whatever the tile.  All matrices column-major.
//
// The Cholesky factorization uses the same kernel for its symmetric update
// A22 -= L21 L21^T: B is then read transposed (TB: element (k, j) at
// B[j + k ldb]) and only the lower triangle is written (lshift >= 0: element
// (i, j) of C is kept when i >= j + lshift, and tiles wholly above that
// diagonal return at once).
#include "common.cuh"
#include "internal.h"

namespace lu {

constexpr int kGK = 16;

template <typename T, int TM, int TN, bool TB>
__global__ void __launch_bounds__((TM / 4) * (TN / 4))
gemm_update_simt(int m, int n, int k, const T *__restrict__ A, int lda, const T *__restrict__ B, int ldb,
                 T *__restrict__ C, int ldc, int lshift, CtaTrace tr) {
    const unsigned long long t_start = tr.ring ? lu_globaltimer() : 0ull;
    constexpr int TX = TM / 4, TY = TN / 4, NT = TX * TY;
    __shared__ T As[kGK][TM];       // As[kk][row]
    __shared__ T Bs[kGK][TN + 1];   // Bs[kk][col]
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int row0 = blockIdx.x * TM, col0 = blockIdx.y * TN;
    if (lshift >= 0 && row0 + TM - 1 < col0 + lshift) return;   // wholly above the kept triangle
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < k; k0 += kGK) {
        // A tile: TM rows x 16 k (coalesced down the rows)
        for (int e = threadIdx.x; e < TM * kGK; e += NT) {
            const int r = e % TM, kk = e / TM;
            const int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < m && gk < k) ? A[(size_t)gr + (size_t)gk * lda] : T(0);
        }
        // B tile: 16 k x TN cols (coalesced down k, or along the columns when transposed)
        for (int e = threadIdx.x; e < TN * kGK; e += NT) {
            const int kk = TB ? e / TN : e % kGK, c = TB ? e % TN : e / kGK;
            const int gc = col0 + c, gk = k0 + kk;
            Bs[kk][c] = (gc < n && gk < k) ? (TB ? B[(size_t)gc + (size_t)gk * ldb] : B[(size_t)gk + (size_t)gc * ldb]) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + TX * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][ty + TY * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gc = col0 + ty + TY * j;
        if (gc >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gr = row0 + tx + TX * i;
            if (gr < m && (lshift < 0 || gr >= gc + lshift)) {
                T *c = &C[(size_t)gr + (size_t)gc * ldc];
                *c = *c - acc[i][j];
            }
        }
    }
    if (threadIdx.x == 0) lu_trace_cta(tr, t_start, 1);
}

template <typename T>
cudaError_t launch_gemm_simt(int m, int n, int k, const T *A, int lda, const T *B, int ldb, T *C, int ldc,
                             cudaStream_t s, CtaTrace tr, bool transb, int lshift, int tile) {
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    int sms = 0;
    cudaError_t e = lu_sm_count(&sms);
    if (e != cudaSuccess) return e;
    // tile 1: 64 x 64 tiles, 2: 32 x 32, 0: 64 x 64 when that makes at least one tile per SM
    // (both shapes accumulate in the same order: the same bits)
    const long long big = (long long)lu_ceil_div(m, 64) * lu_ceil_div(n, 64);
    if (tile == 1 || (tile != 2 && big >= sms)) {
        dim3 grid(lu_ceil_div(m, 64), lu_ceil_div(n, 64));
        if (grid.y > 65535) return cudaErrorInvalidValue;
        if (transb)
            gemm_update_simt<T, 64, 64, true><<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, lshift, tr);
        else
            gemm_update_simt<T, 64, 64, false><<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, lshift, tr);
    } else {
        dim3 grid(lu_ceil_div(m, 32), lu_ceil_div(n, 32));
        if (transb)
            gemm_update_simt<T, 32, 32, true><<<grid, 64, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, lshift, tr);
        else
            gemm_update_simt<T, 32, 32, false><<<grid, 64, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, lshift, tr);
    }
    lu_count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_gemm_simt<double>(int, int, int, const double *, int, const double *, int, double *, int, cudaStream_t,
                                              CtaTrace, bool, int, int);
template cudaError_t launch_gemm_simt<float>(int, int, int, const float *, int, const float *, int, float *, int, cudaStream_t,
                                             CtaTrace, bool, int, int);

}  // namespace lu
