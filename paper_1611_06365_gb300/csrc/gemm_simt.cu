// Trailing update RL3 / PF2 / RU2 on CUDA cores: C := C - A * B
// (section 3.1, Figure 1 right; section 3.2, Figure 3).
//
// FP64 on GB300 runs at the same rate on DFMA and on the legacy DMMA path
// (about 1 TFLOP/s for the whole GPU), and the update's arithmetic intensity
// (2b/16 flop/byte for b >= 8) is far above the FP64 machine balance, so a
// register-tiled DFMA kernel is bound by the FP64 pipe, not by memory.  The
// same kernel in FP32 serves the FP32-native factorization.
//
// Tile 64 x 64 per CTA, 256 threads, 4 x 4 outputs per thread, K staged
// through shared memory in chunks of 16.  All matrices column-major.
#include "common.cuh"

namespace lu {

constexpr int kGT = 64, kGK = 16, kGThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kGThreads)
gemm_update_simt(int m, int n, int k, const T *__restrict__ A, int lda, const T *__restrict__ B, int ldb,
                 T *__restrict__ C, int ldc) {
    __shared__ T As[kGK][kGT];       // As[kk][row]
    __shared__ T Bs[kGK][kGT + 1];   // Bs[kk][col]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.x * kGT, col0 = blockIdx.y * kGT;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < k; k0 += kGK) {
        // A tile: 64 rows x 16 k (coalesced down the rows)
        for (int e = threadIdx.x; e < kGT * kGK; e += kGThreads) {
            const int r = e & (kGT - 1), kk = e / kGT;
            const int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < m && gk < k) ? A[(size_t)gr + (size_t)gk * lda] : T(0);
        }
        // B tile: 16 k x 64 cols (coalesced down k)
        for (int e = threadIdx.x; e < kGT * kGK; e += kGThreads) {
            const int kk = e & (kGK - 1), c = e / kGK;
            const int gc = col0 + c, gk = k0 + kk;
            Bs[kk][c] = (gc < n && gk < k) ? B[(size_t)gk + (size_t)gc * ldb] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gc = col0 + ty + 16 * j;
        if (gc >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gr = row0 + tx + 16 * i;
            if (gr < m) {
                T *c = &C[(size_t)gr + (size_t)gc * ldc];
                *c = *c - acc[i][j];
            }
        }
    }
}

template <typename T>
cudaError_t launch_gemm_simt(int m, int n, int k, const T *A, int lda, const T *B, int ldb, T *C, int ldc,
                             cudaStream_t s) {
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    dim3 grid(lu_ceil_div(m, kGT), lu_ceil_div(n, kGT));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    gemm_update_simt<T><<<grid, kGThreads, 0, s>>>(m, n, k, A, lda, B, ldb, C, ldc);
    lu_count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_gemm_simt<double>(int, int, int, const double *, int, const double *, int, double *, int, cudaStream_t);
template cudaError_t launch_gemm_simt<float>(int, int, int, const float *, int, const float *, int, float *, int, cudaStream_t);

}  // namespace lu
