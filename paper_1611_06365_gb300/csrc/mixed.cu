// Kernels of the mixed-precision solve (the precision ladder is not part of
// the paper; it refines the FP32 factorization of the blocked look-ahead LU):
//
//   cast_rowsum   A32 := fl32(A) and the row sums of |A| (for ||A||_inf);
//   residual      R := B - A X in FP64, column chunks summed in a fixed order
//                 (deterministic), reading FP64 A once;
//   absmax        ||v||_inf of each column (atomicMax on the IEEE bit
//                 pattern, which orders non-negative doubles);
//   to_f32_scaled / axpy_scaled  the scaled FP32 correction solve glue.
#include "common.cuh"
#include "internal.h"
#include <algorithm>

namespace lu {

constexpr int kRowTile = 256;
constexpr int kColChunk = 256;
constexpr int kRhsPass = 16;

__global__ void cast_rowsum_kernel(int n, const double *__restrict__ A, int lda, float *__restrict__ A32, int lda32,
                                   double *__restrict__ rowsum) {
    const int i = blockIdx.x * kRowTile + threadIdx.x;
    const int j0 = blockIdx.y * kColChunk, j1 = min(n, j0 + kColChunk);
    if (i >= n) return;
    double s = 0.0;
    for (int j = j0; j < j1; ++j) {
        const double a = A[(size_t)i + (size_t)j * lda];
        A32[(size_t)i + (size_t)j * lda32] = (float)a;
        s += fabs(a);
    }
    atomicAdd(&rowsum[i], s);
}

__global__ void residual_partial_kernel(int n, int nrhs, const double *__restrict__ A, int lda,
                                        const double *__restrict__ X, int ldx, double *__restrict__ part) {
    __shared__ double xs[kColChunk][kRhsPass];
    const int i = blockIdx.x * kRowTile + threadIdx.x;
    const int j0 = blockIdx.y * kColChunk, j1 = min(n, j0 + kColChunk);
    for (int q0 = 0; q0 < nrhs; q0 += kRhsPass) {
        const int nq = min(kRhsPass, nrhs - q0);
        __syncthreads();
        for (int e = threadIdx.x; e < (j1 - j0) * nq; e += blockDim.x)
            xs[e % (j1 - j0)][e / (j1 - j0)] = X[(size_t)(j0 + e % (j1 - j0)) + (size_t)(q0 + e / (j1 - j0)) * ldx];
        __syncthreads();
        if (i < n) {
            double acc[kRhsPass];
#pragma unroll
            for (int q = 0; q < kRhsPass; ++q) acc[q] = 0.0;
            if (nq == 1) {
                for (int j = j0; j < j1; ++j) acc[0] = fma(A[(size_t)i + (size_t)j * lda], xs[j - j0][0], acc[0]);
            } else {
                for (int j = j0; j < j1; ++j) {
                    const double a = A[(size_t)i + (size_t)j * lda];
#pragma unroll
                    for (int q = 0; q < kRhsPass; ++q)
                        if (q < nq) acc[q] = fma(a, xs[j - j0][q], acc[q]);
                }
            }
            for (int q = 0; q < nq; ++q) part[((size_t)blockIdx.y * nrhs + q0 + q) * n + i] = acc[q];
        }
    }
}

__global__ void residual_finish_kernel(int n, int nrhs, int nchunks, const double *__restrict__ part,
                                       const double *__restrict__ B, int ldb, double *__restrict__ R, int ldr,
                                       unsigned long long *__restrict__ rmax) {
    const size_t total = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += part[((size_t)c * nrhs + q) * n + i];
        const double r = B ? B[(size_t)i + (size_t)q * ldb] - s : s;   // no B: the product A X itself
        R[(size_t)i + (size_t)q * ldr] = r;
        atomicMax(&rmax[q], (unsigned long long)__double_as_longlong(fabs(r)));
    }
}

__global__ void absmax_kernel(int n, int nrhs, const double *__restrict__ V, int ldv, unsigned long long *__restrict__ out) {
    const size_t total = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        atomicMax(&out[q], (unsigned long long)__double_as_longlong(fabs(V[(size_t)i + (size_t)q * ldv])));
    }
}

__global__ void vecmax_kernel(int n, const double *__restrict__ v, unsigned long long *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicMax(out, (unsigned long long)__double_as_longlong(v[i]));
}

// R32 := fl32(R / s_q) for column q, s_q = ||r_q||_inf (1 when zero)
__global__ void to_f32_scaled_kernel(int n, int nrhs, const double *__restrict__ R, int ldr,
                                     const unsigned long long *__restrict__ rmax, float *__restrict__ R32, int ldr32) {
    const size_t total = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        double s = __longlong_as_double((long long)rmax[q]);
        if (!(s > 0.0) || isinf(s)) s = 1.0;
        R32[(size_t)i + (size_t)q * ldr32] = (float)(R[(size_t)i + (size_t)q * ldr] / s);
    }
}

// X += s_q * D32
__global__ void axpy_scaled_kernel(int n, int nrhs, const float *__restrict__ D32, int ldd,
                                   const unsigned long long *__restrict__ rmax, double *__restrict__ X, int ldx) {
    const size_t total = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        double s = __longlong_as_double((long long)rmax[q]);
        if (!(s > 0.0) || isinf(s)) s = 1.0;
        X[(size_t)i + (size_t)q * ldx] += s * (double)D32[(size_t)i + (size_t)q * ldd];
    }
}

// out[q] = bits of max_i |s_q D32(i, q)|: the size of the correction axpy_scaled adds
__global__ void absmax_scaled_f32_kernel(int n, int nrhs, const float *__restrict__ D32, int ldd,
                                         const unsigned long long *__restrict__ rmax, unsigned long long *__restrict__ out) {
    const size_t total = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        double s = __longlong_as_double((long long)rmax[q]);
        if (!(s > 0.0) || isinf(s)) s = 1.0;
        atomicMax(&out[q], (unsigned long long)__double_as_longlong(fabs(s * (double)D32[(size_t)i + (size_t)q * ldd])));
    }
}

__global__ void axpy_f64_kernel(int n, int nrhs, const double *__restrict__ D, int ldd, double *__restrict__ X, int ldx) {
    const size_t total = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), q = (int)(e / n);
        X[(size_t)i + (size_t)q * ldx] += D[(size_t)i + (size_t)q * ldd];
    }
}

static int grid_for(size_t total) { return (int)std::min<size_t>((total + 255) / 256, 152 * 16); }

cudaError_t launch_cast_rowsum(int n, const double *A, int lda, float *A32, int lda32, double *rowsum, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(rowsum, 0, sizeof(double) * n, s);
    if (e != cudaSuccess) return e;
    dim3 grid(lu_ceil_div(n, kRowTile), lu_ceil_div(n, kColChunk));
    cast_rowsum_kernel<<<grid, kRowTile, 0, s>>>(n, A, lda, A32, lda32, rowsum);
    lu_count_launch();
    return cudaGetLastError();
}

size_t residual_workspace_doubles(int n, int nrhs) { return (size_t)lu_ceil_div(n, kColChunk) * nrhs * n; }

cudaError_t launch_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B, int ldb,
                            double *R, int ldr, double *part, unsigned long long *rmax, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(rmax, 0, sizeof(unsigned long long) * nrhs, s);
    if (e != cudaSuccess) return e;
    const int nchunks = lu_ceil_div(n, kColChunk);
    dim3 grid(lu_ceil_div(n, kRowTile), nchunks);
    residual_partial_kernel<<<grid, kRowTile, 0, s>>>(n, nrhs, A, lda, X, ldx, part);
    lu_count_launch();
    residual_finish_kernel<<<grid_for((size_t)n * nrhs), 256, 0, s>>>(n, nrhs, nchunks, part, B, ldb, R, ldr, rmax);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_axpy_f64(int n, int nrhs, const double *D, int ldd, double *X, int ldx, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    axpy_f64_kernel<<<grid_for((size_t)n * nrhs), 256, 0, s>>>(n, nrhs, D, ldd, X, ldx);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_absmax(int n, int nrhs, const double *V, int ldv, unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long) * nrhs, s);
    if (e != cudaSuccess || n <= 0) return e;
    absmax_kernel<<<grid_for((size_t)n * nrhs), 256, 0, s>>>(n, nrhs, V, ldv, out);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_absmax_scaled_f32(int n, int nrhs, const float *D32, int ldd, const unsigned long long *rmax,
                                     unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long) * nrhs, s);
    if (e != cudaSuccess || n <= 0) return e;
    absmax_scaled_f32_kernel<<<grid_for((size_t)n * nrhs), 256, 0, s>>>(n, nrhs, D32, ldd, rmax, out);
    lu_count_launch();
    return cudaGetLastError();
}

// R32 := n values uniform in [-1, 1) from a counter hash of (seed, i): splitmix64
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014), top 24 bits.  The right-hand side of the condition estimate.
__global__ void fill_probe_kernel(int n, unsigned long long seed, float *__restrict__ R32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        R32[i] = (float)(z >> 40) * 0x1p-23f - 1.0f;
    }
}

cudaError_t launch_fill_probe(int n, unsigned long long seed, float *R32, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    fill_probe_kernel<<<grid_for(n), 256, 0, s>>>(n, seed, R32);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_vecmax(int n, const double *v, unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n <= 0) return e;
    vecmax_kernel<<<grid_for(n), 256, 0, s>>>(n, v, out);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_to_f32_scaled(int n, int nrhs, const double *R, int ldr, const unsigned long long *rmax, float *R32,
                                 int ldr32, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    to_f32_scaled_kernel<<<grid_for((size_t)n * nrhs), 256, 0, s>>>(n, nrhs, R, ldr, rmax, R32, ldr32);
    lu_count_launch();
    return cudaGetLastError();
}

cudaError_t launch_axpy_scaled(int n, int nrhs, const float *D32, int ldd, const unsigned long long *rmax, double *X,
                               int ldx, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    axpy_scaled_kernel<<<grid_for((size_t)n * nrhs), 256, 0, s>>>(n, nrhs, D32, ldd, rmax, X, ldx);
    lu_count_launch();
    return cudaGetLastError();
}

}  // namespace lu
