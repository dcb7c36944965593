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
#include "common.cuh"

namespace lu {

constexpr int kGK = 16;

template <typename T, int TM, int TN>
__global__ void __launch_bounds__((TM / 4) * (TN / 4))
gemm_update_simt(int m, int n, int k, const T *__restrict__ A, int lda, const T *__restrict__ B, int ldb,
                 T *__restrict__ C, int ldc, CtaTrace tr) {
    const unsigned long long t_start = tr.ring ? lu_globaltimer() : 0ull;
    constexpr int TX = TM / 4, TY = TN / 4, NT = TX * TY;
    __shared__ T As[kGK][TM];       // As[kk][row]
    __shared__ T Bs[kGK][TN + 1];   // Bs[kk][col]
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int row0 = blockIdx.x * TM, col0 = blockIdx.y * TN;
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
        // B tile: 16 k x TN cols (coalesced down k)
        for (int e = threadIdx.x; e < TN * kGK; e += NT) {
            const int kk = e % kGK, c = e / kGK;
            const int gc = col0 + c, gk = k0 + kk;
            Bs[kk][c] = (gc < n && gk < k) ? B[(size_t)gk + (size_t)gc * ldb] : T(0);
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
            if (gr < m) {
                T *c = &C[(size_t)gr + (size_t)gc * ldc];
                *c = *c - acc[i][j];
            }
        }
    }
    if (threadIdx.x == 0) lu_trace_cta(tr, t_start, 1);
}

template <typename T>
cudaError_t launch_gemm_simt(int m, int n, int k, const T *A, int lda, const T *B, int ldb, T *C, int ldc,
                             cudaStream_t s, CtaTrace tr) {
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    static int sms = 0;
    if (!sms) {
        int d = 0;
        cudaError_t e = cudaGetDevice(&d);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        if (e != cudaSuccess) return e;
    }
    const long long big = (long long)lu_ceil_div(m, 64) * lu_ceil_div(n, 64);
    if (big >= sms) {
        dim3 grid(lu_ceil_div(m, 64), lu_ceil_div(n, 64));
        if (grid.y > 65535) return cudaErrorInvalidValue;
        gemm_update_simt<T, 64, 64><<<grid, 256, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, tr);
    } else {
        dim3 grid(lu_ceil_div(m, 32), lu_ceil_div(n, 32));
        gemm_update_simt<T, 32, 32><<<grid, 64, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc, tr);
    }
    lu_count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_gemm_simt<double>(int, int, int, const double *, int, const double *, int, double *, int, cudaStream_t,
                                              CtaTrace);
template cudaError_t launch_gemm_simt<float>(int, int, int, const float *, int, const float *, int, float *, int, cudaStream_t,
                                             CtaTrace);

}  // namespace lu
