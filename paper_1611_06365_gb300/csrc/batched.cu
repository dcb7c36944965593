// Batched LU with partial pivoting and solve: one CTA per matrix, all
// matrices of a batch in one launch (orders may differ).
//
// Each CTA runs the unblocked right-looking algorithm of section 3.1
// (Figure 1, left) with partial pivoting on its matrix: per column, a
// block-wide (|a|, row) argmax (warp shuffles, smallest row on ties), the row
// interchange over all columns, IEEE division of the column below the
// diagonal, and the rank-1 update of the trailing block.  A matrix whose
// n^2 entries fit in the CTA's shared memory is factored there (read once,
// written once); larger ones are factored in place in global memory, where
// the L2 cache holds them.
#include "common.cuh"
#include "internal.h"
#include <climits>

namespace lu {

constexpr int kBThreads = 256;

template <typename T>
__device__ __forceinline__ void block_argmax(T &mag, int &idx, T *red_m, int *red_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T m2 = __shfl_xor_sync(0xffffffffu, mag, o);
        int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (lu_better(m2, i2, mag, idx)) { mag = m2; idx = i2; }
    }
    if (lane == 0) { red_m[warp] = mag; red_i[warp] = idx; }
    __syncthreads();
    if (warp == 0) {
        mag = lane < kBThreads / 32 ? red_m[lane] : T(-1);
        idx = lane < kBThreads / 32 ? red_i[lane] : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T m2 = __shfl_xor_sync(0xffffffffu, mag, o);
            int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
            if (lu_better(m2, i2, mag, idx)) { mag = m2; idx = i2; }
        }
        if (lane == 0) { red_m[0] = mag; red_i[0] = idx; }
    }
    __syncthreads();
    mag = red_m[0];
    idx = red_i[0];
    __syncthreads();
}

// Factor the n x n matrix M (leading dimension ld; shared or global memory).
template <typename T>
__device__ int getf2_block(T *M, int ld, int n, int *ipiv, T *red_m, int *red_i) {
    int info = 0;
    for (int j = 0; j < n; ++j) {
        T best = T(-1);
        int bidx = INT_MAX;
        for (int i = j + threadIdx.x; i < n; i += kBThreads) {
            T v = lu_abs(M[i + (size_t)j * ld]);
            if (lu_better(v, i, best, bidx)) { best = v; bidx = i; }
        }
        block_argmax(best, bidx, red_m, red_i);
        const int p = (bidx == INT_MAX) ? j : bidx;
        const T piv = M[p + (size_t)j * ld];
        if (threadIdx.x == 0) ipiv[j] = p + 1;
        if (piv == T(0)) {
            if (info == 0) info = j + 1;
            __syncthreads();
            continue;
        }
        if (p != j)
            for (int c = threadIdx.x; c < n; c += kBThreads) {
                T t = M[j + (size_t)c * ld];
                M[j + (size_t)c * ld] = M[p + (size_t)c * ld];
                M[p + (size_t)c * ld] = t;
            }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < n; i += kBThreads) M[i + (size_t)j * ld] = M[i + (size_t)j * ld] / piv;
        __syncthreads();
        const int mm = n - j - 1;
        for (int e = threadIdx.x; e < mm * mm; e += kBThreads) {
            const int i = j + 1 + e % mm, c = j + 1 + e / mm;
            M[i + (size_t)c * ld] = fma(-M[i + (size_t)j * ld], M[j + (size_t)c * ld], M[i + (size_t)c * ld]);
        }
        __syncthreads();
    }
    return info;
}

template <typename T>
__global__ void __launch_bounds__(kBThreads)
getrf_batched_kernel(const int *__restrict__ ns, T *const *__restrict__ As, const int *__restrict__ ldas,
                     int *const *__restrict__ ipivs, int *__restrict__ infos, int smem_elems) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T red_m[32];
    __shared__ int red_i[32];
    const int t = blockIdx.x;
    const int n = ns[t], lda = ldas[t];
    T *A = As[t];
    int *ipiv = ipivs[t];
    int info = 0;
    if (n > 0) {
        if (n * n <= smem_elems) {
            T *S = reinterpret_cast<T *>(smem_raw);
            for (int e = threadIdx.x; e < n * n; e += kBThreads) S[e] = A[(e % n) + (size_t)(e / n) * lda];
            __syncthreads();
            info = getf2_block(S, n, n, ipiv, red_m, red_i);
            for (int e = threadIdx.x; e < n * n; e += kBThreads) A[(e % n) + (size_t)(e / n) * lda] = S[e];
        } else {
            info = getf2_block(A, lda, n, ipiv, red_m, red_i);
        }
    }
    if (threadIdx.x == 0) infos[t] = info;
}

// X := A^{-1} B for each member: interchanges in order, then unit lower and
// upper substitution (the factors stay where they are; B in shared memory).
template <typename T>
__global__ void __launch_bounds__(kBThreads)
getrs_batched_kernel(int nrhs, const int *__restrict__ ns, const T *const *__restrict__ LUs, const int *__restrict__ ldas,
                     const int *const *__restrict__ ipivs, T *const *__restrict__ Bs, const int *__restrict__ ldbs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *x = reinterpret_cast<T *>(smem_raw);
    const int t = blockIdx.x;
    const int n = ns[t], lda = ldas[t], ldb = ldbs[t];
    const T *LU = LUs[t];
    const int *ipiv = ipivs[t];
    T *B = Bs[t];
    for (int q = 0; q < nrhs; ++q) {
        for (int i = threadIdx.x; i < n; i += kBThreads) x[i] = B[i + (size_t)q * ldb];
        __syncthreads();
        if (threadIdx.x == 0)
            for (int j = 0; j < n; ++j) {
                const int p = ipiv[j] - 1;
                if (p != j) { T tmp = x[j]; x[j] = x[p]; x[p] = tmp; }
            }
        __syncthreads();
        for (int j = 0; j < n; ++j) {
            const T y = x[j];
            for (int i = j + 1 + threadIdx.x; i < n; i += kBThreads) x[i] = fma(-LU[i + (size_t)j * lda], y, x[i]);
            __syncthreads();
        }
        for (int j = n - 1; j >= 0; --j) {
            if (threadIdx.x == 0) x[j] = x[j] / LU[j + (size_t)j * lda];
            __syncthreads();
            const T y = x[j];
            for (int i = threadIdx.x; i < j; i += kBThreads) x[i] = fma(-LU[i + (size_t)j * lda], y, x[i]);
            __syncthreads();
        }
        for (int i = threadIdx.x; i < n; i += kBThreads) B[i + (size_t)q * ldb] = x[i];
        __syncthreads();
    }
}

template <typename T>
cudaError_t launch_getrf_batched(int batch, const int *ns, T *const *As, const int *ldas, int *const *ipivs, int *infos,
                                 int max_n, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    const size_t cap = 200 * 1024;
    size_t need = (size_t)max_n * max_n * sizeof(T);
    size_t smem = need <= cap ? need : 0;
    if (smem == 0) {
        // the largest members run in global memory; keep shared memory for the rest
        smem = cap;
    }
    cudaError_t e = cudaFuncSetAttribute(getrf_batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    getrf_batched_kernel<T><<<batch, kBThreads, smem, s>>>(ns, As, ldas, ipivs, infos, (int)(smem / sizeof(T)));
    lu_count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_getrs_batched(int batch, int nrhs, const int *ns, const T *const *LUs, const int *ldas,
                                 const int *const *ipivs, T *const *Bs, const int *ldbs, int max_n, cudaStream_t s) {
    if (batch <= 0 || nrhs <= 0) return cudaSuccess;
    size_t smem = (size_t)max_n * sizeof(T);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(getrs_batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    getrs_batched_kernel<T><<<batch, kBThreads, smem, s>>>(nrhs, ns, LUs, ldas, ipivs, Bs, ldbs);
    lu_count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_getrf_batched<double>(int, const int *, double *const *, const int *, int *const *, int *, int, cudaStream_t);
template cudaError_t launch_getrf_batched<float>(int, const int *, float *const *, const int *, int *const *, int *, int, cudaStream_t);
template cudaError_t launch_getrs_batched<double>(int, int, const int *, const double *const *, const int *, const int *const *, double *const *, const int *, int, cudaStream_t);
template cudaError_t launch_getrs_batched<float>(int, int, const int *, const float *const *, const int *, const int *const *, float *const *, const int *, int, cudaStream_t);

}  // namespace lu
