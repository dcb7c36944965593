// Triangular solves with the LU factors (getrs): X := U^{-1} L^{-1} P B.
//
// * ipiv_to_perm: the sequential interchanges of ipiv (LAPACK meaning) turned
//   into the permutation vector perm (P B row j = B row perm[j]), 64
//   interchanges at a time with the same row-map construction as the
//   factorization's interchange kernel.
// * gather_rows: X = B[perm, :].
// * trsv_blocks: blocked substitution by row blocks of 64.  A persistent grid
//   takes row blocks in order from an atomic ticket; the CTA of block I reads
//   the off-diagonal blocks of its rows as the solutions of earlier blocks
//   are published (flag per block, release/acquire), then solves its diagonal
//   block and publishes.  A CTA only waits for blocks handed out before its
//   own, which belong to CTAs already running, so the chain always advances;
//   every wait is bounded and records LU_ERR_TIMEOUT on expiry.
#include "common.cuh"
#include <algorithm>

namespace lu {

constexpr int kTB = 64;           // row block
constexpr int kTThreads = 256;
constexpr int kMaxRhs = 16;       // right-hand sides per pass
constexpr int kHash = 1024;

__global__ void ipiv_to_perm_kernel(const int *__restrict__ ipiv, int n, int *__restrict__ perm) {
    __shared__ int keys[kHash], slot_of[kHash];
    __shared__ int rows[2 * 64], cont[2 * 64], vals[2 * 64];
    __shared__ int cnt_s;
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = i;
    __syncthreads();
    for (int kb = 0; kb < n; kb += 64) {
        const int b = min(64, n - kb);
        for (int i = threadIdx.x; i < kHash; i += blockDim.x) keys[i] = -1;
        for (int t = threadIdx.x; t < b; t += blockDim.x) { rows[t] = kb + t; cont[t] = kb + t; }
        __syncthreads();
        if (threadIdx.x == 0) {
            int cnt = b;
            for (int j = 0; j < b; ++j) {
                const int r = kb + j, p = ipiv[kb + j] - 1;
                if (p == r) continue;
                int ip;
                if (p < kb + b) {
                    ip = p - kb;
                } else {
                    unsigned h = ((unsigned)p * 2654435761u) & (kHash - 1);
                    while (keys[h] != -1 && keys[h] != p) h = (h + 1) & (kHash - 1);
                    if (keys[h] == -1) { keys[h] = p; slot_of[h] = cnt; rows[cnt] = p; cont[cnt] = p; ++cnt; }
                    ip = slot_of[h];
                }
                int t = cont[j]; cont[j] = cont[ip]; cont[ip] = t;
            }
            cnt_s = cnt;
        }
        __syncthreads();
        const int cnt = cnt_s;
        for (int s = threadIdx.x; s < cnt; s += blockDim.x) vals[s] = perm[cont[s]];
        __syncthreads();
        for (int s = threadIdx.x; s < cnt; s += blockDim.x) perm[rows[s]] = vals[s];
        __syncthreads();
    }
}

template <typename TI, typename TO>
__global__ void gather_rows_kernel(int n, int nrhs, const int *__restrict__ perm, const TI *__restrict__ B, int ldb,
                                   TO *__restrict__ X, int ldx) {
    const size_t total = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), c = (int)(e / n);
        X[i + (size_t)c * ldx] = (TO)B[perm[i] + (size_t)c * ldb];
    }
}

// LOWER: unit lower forward substitution (blocks taken top-down);
// !LOWER: upper backward substitution (blocks taken bottom-up).
template <typename T, bool LOWER>
__global__ void __launch_bounds__(kTThreads)
trsv_blocks(const T *__restrict__ LU, int lda, int n, int nrhs, T *__restrict__ X, int ldx, int *__restrict__ ticket,
            int *__restrict__ flags, int *__restrict__ status, long long bound_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*Ld)[kTB + 1] = reinterpret_cast<T (*)[kTB + 1]>(smem_raw);                       // diagonal block [r][c]
    T (*yJ)[kMaxRhs] = reinterpret_cast<T (*)[kMaxRhs]>(smem_raw + sizeof(T) * kTB * (kTB + 1));
    T (*part)[kTB][kMaxRhs] = reinterpret_cast<T (*)[kTB][kMaxRhs]>(smem_raw + sizeof(T) * (kTB * (kTB + 1) + kTB * kMaxRhs));
    T (*xb)[kMaxRhs] = reinterpret_cast<T (*)[kMaxRhs]>(smem_raw + sizeof(T) * (kTB * (kTB + 1) + 5 * kTB * kMaxRhs));
    __shared__ int tk_s, abort_s;
    const int nblk = (n + kTB - 1) / kTB;
    const int r = threadIdx.x & (kTB - 1), g = threadIdx.x >> 6;
    for (;;) {
        if (threadIdx.x == 0) { tk_s = atomicAdd(ticket, 1); abort_s = 0; }
        __syncthreads();
        const int t = tk_s;
        if (t >= nblk) break;
        const int I = LOWER ? t : nblk - 1 - t;
        const int r0 = I * kTB, rows = min(kTB, n - r0);
        T acc[kMaxRhs];
#pragma unroll
        for (int q = 0; q < kMaxRhs; ++q) acc[q] = T(0);
        // off-diagonal blocks, in the order their solutions appear
        for (int s = 0; s < (LOWER ? I : nblk - 1 - I); ++s) {
            const int J = LOWER ? s : nblk - 1 - s;
            const int c0 = J * kTB, cols = min(kTB, n - c0);
            if (threadIdx.x == 0) {
                if (!lu_wait_flag(&flags[J], 1, status, bound_ns)) abort_s = 1;
                __threadfence();
            }
            __syncthreads();
            if (abort_s) return;
            for (int e = threadIdx.x; e < cols * nrhs; e += kTThreads) {
                const int c = e % cols, q = e / cols;
                yJ[c][q] = __ldcg(&X[(size_t)(c0 + c) + (size_t)q * ldx]);
            }
            __syncthreads();
            if (r < rows) {
                for (int c = g; c < cols; c += 4) {
                    const T l = LU[(size_t)(r0 + r) + (size_t)(c0 + c) * lda];
                    for (int q = 0; q < nrhs; ++q) acc[q] = fma(-l, yJ[c][q], acc[q]);
                }
            }
            __syncthreads();
        }
        for (int q = 0; q < nrhs; ++q) part[g][r][q] = acc[q];
        // diagonal block into shared memory
        for (int e = threadIdx.x; e < kTB * kTB; e += kTThreads) {
            const int rr = e & (kTB - 1), cc = e >> 6;
            Ld[rr][cc] = (rr < rows && cc < rows) ? LU[(size_t)(r0 + rr) + (size_t)(r0 + cc) * lda] : T(0);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * nrhs; e += kTThreads) {
            const int rr = e % rows, q = e / rows;
            xb[rr][q] = X[(size_t)(r0 + rr) + (size_t)q * ldx] + part[0][rr][q] + part[1][rr][q] + part[2][rr][q] +
                        part[3][rr][q];
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            for (int q = 0; q < nrhs; ++q) {
                if (LOWER) {
                    for (int jj = 0; jj < rows; ++jj) {
                        __syncwarp();
                        const T y = xb[jj][q];
                        for (int rr = lane; rr < rows; rr += 32)
                            if (rr > jj) xb[rr][q] = fma(-Ld[rr][jj], y, xb[rr][q]);
                    }
                } else {
                    for (int jj = rows - 1; jj >= 0; --jj) {
                        __syncwarp();
                        if (lane == 0) xb[jj][q] = xb[jj][q] / Ld[jj][jj];
                        __syncwarp();
                        const T y = xb[jj][q];
                        for (int rr = lane; rr < jj; rr += 32) xb[rr][q] = fma(-Ld[rr][jj], y, xb[rr][q]);
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * nrhs; e += kTThreads) {
            const int rr = e % rows, q = e / rows;
            X[(size_t)(r0 + rr) + (size_t)q * ldx] = xb[rr][q];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            lu_st_release(&flags[I], 1);
        }
    }
}

cudaError_t launch_ipiv_to_perm(const int *ipiv, int n, int *perm, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    ipiv_to_perm_kernel<<<1, 256, 0, s>>>(ipiv, n, perm);
    lu_count_launch();
    return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_gather_rows(int n, int nrhs, const int *perm, const TI *B, int ldb, TO *X, int ldx, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    size_t total = (size_t)n * nrhs;
    int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 8);
    gather_rows_kernel<TI, TO><<<grid, 256, 0, s>>>(n, nrhs, perm, B, ldb, X, ldx);
    lu_count_launch();
    return cudaGetLastError();
}

// Workspace: ints [2 + 2*nblk] (two tickets, two flag arrays), zeroed here.
template <typename T>
cudaError_t launch_trsv_pair(const T *LU, int lda, int n, int nrhs, T *X, int ldx, int *ws, int *status,
                             long long bound_ns, int sms, cudaStream_t s) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    const int nblk = (n + kTB - 1) / kTB;
    cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(int) * (size_t)(2 + 2 * nblk), s);
    if (e != cudaSuccess) return e;
    const int grid = std::min(nblk, 2 * sms);
    const size_t smem = sizeof(T) * (kTB * (kTB + 1) + 6 * kTB * kMaxRhs);
    e = cudaFuncSetAttribute(trsv_blocks<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(trsv_blocks<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int q0 = 0; q0 < nrhs; q0 += kMaxRhs) {
        const int nq = std::min(kMaxRhs, nrhs - q0);
        if (q0 > 0) {
            e = cudaMemsetAsync(ws, 0, sizeof(int) * (size_t)(2 + 2 * nblk), s);
            if (e != cudaSuccess) return e;
        }
        trsv_blocks<T, true><<<grid, kTThreads, smem, s>>>(LU, lda, n, nq, X + (size_t)q0 * ldx, ldx, ws, ws + 2, status, bound_ns);
        lu_count_launch();
        trsv_blocks<T, false><<<grid, kTThreads, smem, s>>>(LU, lda, n, nq, X + (size_t)q0 * ldx, ldx, ws + 1, ws + 2 + nblk, status, bound_ns);
        lu_count_launch();
    }
    return cudaGetLastError();
}

__global__ void iota_kernel(int *v, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}

cudaError_t launch_iota(int *v, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    iota_kernel<<<std::min(lu_ceil_div(n, 256), 1024), 256, 0, s>>>(v, n);
    lu_count_launch();
    return cudaGetLastError();
}

size_t trsv_workspace_ints(int n) { return (size_t)(2 + 2 * ((n + kTB - 1) / kTB)); }

template cudaError_t launch_gather_rows<double, double>(int, int, const int *, const double *, int, double *, int, cudaStream_t);
template cudaError_t launch_gather_rows<float, float>(int, int, const int *, const float *, int, float *, int, cudaStream_t);
template cudaError_t launch_trsv_pair<double>(const double *, int, int, int, double *, int, int *, int *, long long, int, cudaStream_t);
template cudaError_t launch_trsv_pair<float>(const float *, int, int, int, float *, int, int *, int *, long long, int, cudaStream_t);

}  // namespace lu
