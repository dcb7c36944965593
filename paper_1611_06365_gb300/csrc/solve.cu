// Triangular solves with the LU factors (getrs): X := U^{-1} L^{-1} P B.
//
// * ipiv_to_perm: the sequential interchanges of ipiv (LAPACK meaning) turned
//   into the permutation vector perm (P B row j = B row perm[j]), 64
//   interchanges at a time with the same row-map construction as the
//   factorization's interchange kernel.
// * gather_rows: X = B[perm, :].
// * trsv_blocks: blocked substitution by row blocks of 64.  Warps take row
//   blocks in order from an atomic ticket; the warp of block I accumulates the
//   off-diagonal products of its rows as the solutions of earlier blocks are
//   published, then solves its diagonal block and publishes.  A solution value
//   is published as a tagged 64-bit word (32 value bits + a 32-bit pass tag,
//   two words for a double), so a reader polls the data itself: a word is
//   valid exactly when its tag matches, with no flag, fence or second load on
//   the block-to-block chain.  A warp only waits for blocks handed out before
//   its own, which belong to warps already running, so the chain always
//   advances; every wait is bounded and records LU_ERR_TIMEOUT on expiry.
#include "common.cuh"
#include "internal.h"
#include <algorithm>
#include <atomic>

namespace lu {

constexpr int kTB = 64;           // row block
constexpr int kMaxRhs = 16;       // right-hand sides per pass
constexpr int kHash = 1024;
constexpr int kFlagPad = 32;      // one ticket per 128-byte line
constexpr int kTWarps = 2;        // warps per CTA

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

// Tagged words of the published solutions: word w of value v carries 32 bits
// of v (low half first for a double) and the pass tag in its high half.
template <typename T> struct TagWords { static constexpr int value = sizeof(T) / 4; };

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_word(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void put_tagged(unsigned long long *w, float v, unsigned tag) {
    st_word(w, ((unsigned long long)tag << 32) | __float_as_uint(v));
}
__device__ __forceinline__ void put_tagged(unsigned long long *w, double v, unsigned tag) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    st_word(w, ((unsigned long long)tag << 32) | (b & 0xffffffffULL));
    st_word(w + 1, ((unsigned long long)tag << 32) | (b >> 32));
}
// Reads value words; returns false while any word's tag differs.
__device__ __forceinline__ bool get_tagged(const unsigned long long *w, unsigned tag, float &v) {
    const unsigned long long a = ld_word(w);
    v = __uint_as_float((unsigned)a);
    return (unsigned)(a >> 32) == tag;
}
__device__ __forceinline__ bool get_tagged(const unsigned long long *w, unsigned tag, double &v) {
    const unsigned long long a = ld_word(w), b = ld_word(w + 1);
    v = __longlong_as_double((long long)((b << 32) | (a & 0xffffffffULL)));
    return (unsigned)(a >> 32) == tag && (unsigned)(b >> 32) == tag;
}

// LOWER: unit lower forward substitution (blocks taken top-down);
// !LOWER: upper backward substitution (blocks taken bottom-up).
// One warp per 64-row block (two rows per lane), no CTA-wide barriers: a warp
// takes its block from the ticket, loads its right-hand sides and stages its
// diagonal block and the off-diagonal block of its last dependency in shared
// memory while earlier blocks are still being solved, accumulates the products
// of the earlier published blocks straight from global memory (32 columns of
// loads in flight), and so keeps only a shared-memory product, the diagonal
// solve (shuffles) and the publication on the block-to-block chain.  NQ is
// the number of right-hand sides a chain carries (a compile-time bound, so the
// per-lane arrays stay in registers); the nrhs right-hand sides of a pass form
// nchains independent chains of NQ, run side by side, so the block-to-block
// chain stays as short as for one right-hand side.  W holds the tagged
// solution words, row i of right-hand side q at W[(q * n + i) * TagWords].
template <typename T, bool LOWER, int NQ, bool INV = false>
__global__ void __launch_bounds__(32 * kTWarps)
trsv_blocks(const T *__restrict__ LU, int lda, int n, int nrhs, int nchains, T *__restrict__ Xall, int ldx,
            int *__restrict__ ticket, unsigned long long *__restrict__ Wall, unsigned tag, int *__restrict__ status,
            long long bound_ns, const T *__restrict__ Dinv = nullptr) {
    constexpr int TW = TagWords<T>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *Dg = reinterpret_cast<T *>(smem_raw) + (size_t)warp * 2 * kTB * kTB;   // diagonal block [c][r]
    T *Lp = Dg + (size_t)kTB * kTB;                                            // last dependency block [c][r]
    const int nblk = (n + kTB - 1) / kTB;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nblk * nchains) break;
        // tickets interleave the chains, so they advance together and share the
        // matrix blocks they read through L2
        const int ch = t % nchains, tt = t / nchains;
        const int I = LOWER ? tt : nblk - 1 - tt;
        const int nq = min(NQ, nrhs - ch * NQ);   // right-hand sides of this chain
        T *X = Xall + (size_t)ch * NQ * ldx;
        unsigned long long *W = Wall + (size_t)ch * NQ * n * TW;
        const int r0 = I * kTB, rows = min(kTB, n - r0);
        const bool has0 = lane < rows, has1 = lane + 32 < rows;
        // right-hand sides of the block, loaded before any wait
        T x0[NQ], x1[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            x0[q] = (q < nq && has0) ? X[(size_t)(r0 + lane) + (size_t)q * ldx] : T(0);
            x1[q] = (q < nq && has1) ? X[(size_t)(r0 + lane + 32) + (size_t)q * ldx] : T(0);
        }
        const int ndep = LOWER ? I : nblk - 1 - I;
        const int Jlast = LOWER ? I - 1 : I + 1;
        const int clast = Jlast * kTB, ncl = ndep > 0 ? min(kTB, n - clast) : 0;
        // stage the diagonal block (with INV: its inverse, contiguous [c][r]) and the
        // last dependency's block (matrix data only)
        if (INV) {
            const T *src = Dinv + ((size_t)(LOWER ? 0 : nblk) + I) * kTB * kTB;
            for (int e = lane; e < kTB * kTB; e += 32) Dg[e] = src[e];
        }
        for (int blk = INV ? 1 : 0; blk < 2; ++blk) {
            const int cbase = blk == 0 ? r0 : clast, ncol = blk == 0 ? rows : ncl;
            T *dst = blk == 0 ? Dg : Lp;
            for (int cb = 0; cb < ncol; cb += 16) {
                T a[16], b[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int c = cb + u;
                    a[u] = (has0 && c < ncol) ? LU[(size_t)(r0 + lane) + (size_t)(cbase + c) * lda] : T(0);
                    b[u] = (has1 && c < ncol) ? LU[(size_t)(r0 + lane + 32) + (size_t)(cbase + c) * lda] : T(0);
                }
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    dst[(cb + u) * kTB + lane] = a[u];
                    dst[(cb + u) * kTB + lane + 32] = b[u];
                }
            }
        }
        T acc0[NQ], acc1[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) { acc0[q] = T(0); acc1[q] = T(0); }
        bool ok = true;
        for (int s = 0; s < ndep; ++s) {
            const int J = LOWER ? s : nblk - 1 - s;
            const int c0 = J * kTB, cols = min(kTB, n - c0);
            // poll the tagged solution words of block J
            T y0[NQ], y1[NQ];
            {
                unsigned long long t0 = 0;
                unsigned spins = 0;
                for (;;) {
                    bool got = true;
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        y0[q] = T(0);
                        y1[q] = T(0);
                        if (q < nq && lane < cols)
                            got &= get_tagged(W + ((size_t)q * n + c0 + lane) * TW, tag, y0[q]);
                        if (q < nq && lane + 32 < cols)
                            got &= get_tagged(W + ((size_t)q * n + c0 + lane + 32) * TW, tag, y1[q]);
                    }
                    if (__all_sync(0xffffffffu, got)) break;
                    __nanosleep(spins < 16 ? 20 : 100);
                    if ((++spins & 15u) == 0u) {
                        const unsigned long long now = lu_globaltimer();
                        if (t0 == 0) t0 = now;
                        // a warp-uniform decision: every lane leaves the loop together
                        if (__any_sync(0xffffffffu, (long long)(now - t0) > bound_ns)) { ok = false; break; }
                    }
                }
                if (!ok) {
                    if (lane == 0) atomicExch(status, (int)LU_ERR_TIMEOUT);
                    break;
                }
            }
            if (J == Jlast) {
#pragma unroll 8
                for (int c = 0; c < cols; ++c) {
                    const T l0 = Lp[c * kTB + lane], l1 = Lp[c * kTB + lane + 32];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const T yv = __shfl_sync(0xffffffffu, c < 32 ? y0[q] : y1[q], c & 31);
                        acc0[q] = fma(-l0, yv, acc0[q]);
                        acc1[q] = fma(-l1, yv, acc1[q]);
                    }
                }
            } else {
                const T *col = LU + (size_t)c0 * lda + r0;
                for (int cb = 0; cb < cols; cb += 32) {
                    T la[32], lb[32];
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const int c = cb + u;
                        la[u] = (has0 && c < cols) ? col[(size_t)c * lda + lane] : T(0);
                        lb[u] = (has1 && c < cols) ? col[(size_t)c * lda + lane + 32] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            const T yv = __shfl_sync(0xffffffffu, cb == 0 ? y0[q] : y1[q], u);
                            acc0[q] = fma(-la[u], yv, acc0[q]);
                            acc1[q] = fma(-lb[u], yv, acc1[q]);
                        }
                    }
                }
            }
        }
        if (!ok) return;
        // x = b + products, then the diagonal solve (two rows per lane)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            x0[q] += acc0[q];
            x1[q] += acc1[q];
        }
        __syncwarp();
        if (INV) {
            // x := D^{-1} x with the block's inverse: independent products, no chain
            T n0[NQ], n1[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) { n0[q] = T(0); n1[q] = T(0); }
            for (int c = 0; c < rows; ++c) {
                const T d0 = Dg[c * kTB + lane], d1 = Dg[c * kTB + lane + 32];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const T xc = __shfl_sync(0xffffffffu, c < 32 ? x0[q] : x1[q], c & 31);
                    n0[q] = fma(d0, xc, n0[q]);
                    n1[q] = fma(d1, xc, n1[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) { x0[q] = n0[q]; x1[q] = n1[q]; }
        } else if (LOWER) {
            for (int jj = 0; jj < rows; ++jj) {
                const T l0 = Dg[jj * kTB + lane], l1 = Dg[jj * kTB + lane + 32];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const T y = __shfl_sync(0xffffffffu, jj < 32 ? x0[q] : x1[q], jj & 31);
                    if (lane > jj) x0[q] = fma(-l0, y, x0[q]);
                    if (lane + 32 > jj) x1[q] = fma(-l1, y, x1[q]);
                }
            }
        } else {
            // the diagonal of this lane's two rows and its reciprocals, off the chain;
            // the chain divides with lu_div_fast, and a block where any division was
            // outside its safe range is solved again with the IEEE division
            const T d0 = has0 ? Dg[lane * kTB + lane] : T(1), d1 = has1 ? Dg[(lane + 32) * kTB + lane + 32] : T(1);
            const T rc0 = T(1) / d0, rc1 = T(1) / d1;
            const bool ok0 = lu_div_range<T>::in(d0), ok1 = lu_div_range<T>::in(d1);
            T s0[NQ], s1[NQ], p0[NQ], p1[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) { s0[q] = x0[q]; s1[q] = x1[q]; p0[q] = T(0); p1[q] = T(0); }
            for (int jj = rows - 1; jj >= 0; --jj) {
                const T l0 = Dg[jj * kTB + lane], l1 = Dg[jj * kTB + lane + 32];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    if (jj < 32 && lane == jj) {
                        p0[q] = x0[q];
                        x0[q] = lu_div_fast(x0[q], d0, rc0);
                    }
                    if (jj >= 32 && lane + 32 == jj) {
                        p1[q] = x1[q];
                        x1[q] = lu_div_fast(x1[q], d1, rc1);
                    }
                    const T y = __shfl_sync(0xffffffffu, jj < 32 ? x0[q] : x1[q], jj & 31);
                    if (lane < jj) x0[q] = fma(-l0, y, x0[q]);
                    if (lane + 32 < jj) x1[q] = fma(-l1, y, x1[q]);
                }
            }
            // the divisions' operands, checked once after the chain
            bool unsafe = false;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (has0 && !lu_div_safe(p0[q], ok0)) unsafe = true;
                if (has1 && !lu_div_safe(p1[q], ok1)) unsafe = true;
            }
            if (__any_sync(0xffffffffu, unsafe)) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) { x0[q] = s0[q]; x1[q] = s1[q]; }
                for (int jj = rows - 1; jj >= 0; --jj) {
                    const T l0 = Dg[jj * kTB + lane], l1 = Dg[jj * kTB + lane + 32];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        if (jj < 32 && lane == jj) x0[q] = x0[q] / d0;
                        if (jj >= 32 && lane + 32 == jj) x1[q] = x1[q] / d1;
                        const T y = __shfl_sync(0xffffffffu, jj < 32 ? x0[q] : x1[q], jj & 31);
                        if (lane < jj) x0[q] = fma(-l0, y, x0[q]);
                        if (lane + 32 < jj) x1[q] = fma(-l1, y, x1[q]);
                    }
                }
            }
        }
        // publish the tagged words first (the chain), then the plain result
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (q < nq) {
                if (has0) put_tagged(W + ((size_t)q * n + r0 + lane) * TW, x0[q], tag);
                if (has1) put_tagged(W + ((size_t)q * n + r0 + lane + 32) * TW, x1[q], tag);
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (q < nq) {
                if (has0) X[(size_t)(r0 + lane) + (size_t)q * ldx] = x0[q];
                if (has1) X[(size_t)(r0 + lane + 32) + (size_t)q * ldx] = x1[q];
            }
        }
    }
}

// The same permutation by the plain sequential scan, with the row contents
// (cont[i]: the original row now at position i) in shared memory: one thread
// applies the interchanges in order; the others stage the next chunk of
// ipiv.  n + kPermChunk ints of shared memory.
constexpr int kPermChunk = 2048;
__global__ void __launch_bounds__(1024) ipiv_to_perm_smem(const int *__restrict__ ipiv, int n, int *__restrict__ perm) {
    extern __shared__ int psm[];
    int *cont = psm, *pv = psm + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cont[i] = i;
    for (int c0 = 0; c0 < n; c0 += kPermChunk) {
        const int cn = min(kPermChunk, n - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cn; i += blockDim.x) pv[i] = ipiv[c0 + i] - 1;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int j = 0; j < cn; ++j) {
                const int p = pv[j], jj = c0 + j;
                if (p != jj) {
                    const int t = cont[jj];
                    cont[jj] = cont[p];
                    cont[p] = t;
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = cont[i];
}

cudaError_t launch_ipiv_to_perm(const int *ipiv, int n, int *perm, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(int) * ((size_t)n + kPermChunk);
    if (smem <= 220 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(ipiv_to_perm_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ipiv_to_perm_smem<<<1, 1024, smem, s>>>(ipiv, n, perm);
    } else {
        ipiv_to_perm_kernel<<<1, 256, 0, s>>>(ipiv, n, perm);
    }
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

// Two tickets (one 128-byte line each), then the tagged solution words: up
// to kMaxRhs right-hand sides of n values, two 64-bit words per value (the
// FP64 size; FP32 uses half).
size_t trsv_workspace_ints(int n, int nrhs) {
    const size_t q = (size_t)std::max(1, std::min(nrhs, kMaxRhs));
    return (size_t)2 * kFlagPad + (size_t)4 * q * (size_t)std::max(n, 1);
}

// Inverses of the 64 x 64 diagonal blocks of the factors: block I of the unit
// lower factor at Dinv[I], of the upper factor at Dinv[nblk + I], each
// column-major [c][r] and zero outside the block's rows x rows.  One CTA of 64
// threads per block; thread j forms column j by substitution (IEEE division).
template <typename T>
__global__ void __launch_bounds__(kTB) diag_inverse_kernel(const T *__restrict__ LU, int lda, int n, T *__restrict__ Dinv) {
    extern __shared__ __align__(16) unsigned char di_smem[];
    T(*D)[kTB + 1] = reinterpret_cast<T(*)[kTB + 1]>(di_smem);   // D[c][r]
    T(*Xs)[kTB + 1] = D + kTB;                                     // Xs[c][r]: the inverse
    const int nblk = (n + kTB - 1) / kTB;
    const bool lower = blockIdx.x < (unsigned)nblk;
    const int I = lower ? blockIdx.x : blockIdx.x - nblk;
    const int r0 = I * kTB, rows = min(kTB, n - r0), j = threadIdx.x;
    for (int e = j; e < kTB * kTB; e += kTB) {
        const int c = e / kTB, r = e % kTB;
        D[c][r] = (c < rows && r < rows) ? LU[(size_t)(r0 + r) + (size_t)(r0 + c) * lda] : T(0);
        Xs[c][r] = T(0);
    }
    __syncthreads();
    if (j < rows) {
        if (lower) {
            Xs[j][j] = T(1);
            for (int i = j + 1; i < rows; ++i) {
                T acc = T(0);
                for (int k = j; k < i; ++k) acc = fma(-D[k][i], Xs[j][k], acc);
                Xs[j][i] = acc;
            }
        } else {
            Xs[j][j] = T(1) / D[j][j];
            for (int i = j - 1; i >= 0; --i) {
                T acc = T(0);
                for (int k = i + 1; k <= j; ++k) acc = fma(-D[k][i], Xs[j][k], acc);
                Xs[j][i] = acc / D[i][i];
            }
        }
    }
    __syncthreads();
    T *dst = Dinv + (size_t)blockIdx.x * kTB * kTB;
    for (int e = j; e < kTB * kTB; e += kTB) dst[e] = Xs[e / kTB][e % kTB];
}

template <typename T>
size_t trsv_inverse_elems(int n) { return (size_t)2 * lu_ceil_div(std::max(n, 1), kTB) * kTB * kTB; }

template <typename T>
cudaError_t launch_diag_inverse(const T *LU, int lda, int n, T *Dinv, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(T) * 2 * kTB * (kTB + 1);
    cudaError_t e = cudaFuncSetAttribute(diag_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    diag_inverse_kernel<T><<<2 * lu_ceil_div(n, kTB), kTB, smem, s>>>(LU, lda, n, Dinv);
    lu_count_launch();
    return cudaGetLastError();
}

template <typename T, int NQ, bool INV>
static cudaError_t launch_trsv_nq(int grid, size_t smem, const T *LU, int lda, int n, int nq, T *X, int ldx, int *ws,
                                  int *status, long long bound_ns, cudaStream_t s, const T *Dinv) {
    const int nchains = (nq + NQ - 1) / NQ;
    cudaError_t e = cudaFuncSetAttribute(trsv_blocks<T, true, NQ, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(trsv_blocks<T, false, NQ, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    unsigned long long *W = reinterpret_cast<unsigned long long *>(ws + 2 * kFlagPad);
    // the forward pass publishes with tag 1, the backward pass with tag 2 over the
    // same words: a backward reader never mistakes a forward value for its own
    trsv_blocks<T, true, NQ, INV><<<grid, 32 * kTWarps, smem, s>>>(LU, lda, n, nq, nchains, X, ldx, ws, W, 1u, status,
                                                                   bound_ns, Dinv);
    lu_count_launch();
    trsv_blocks<T, false, NQ, INV><<<grid, 32 * kTWarps, smem, s>>>(LU, lda, n, nq, nchains, X, ldx, ws + kFlagPad, W,
                                                                    2u, status, bound_ns, Dinv);
    lu_count_launch();
    return cudaGetLastError();
}

// CTAs of the substitution kernel resident per SM (shared memory bound).
template <typename T, bool INV>
static int trsv_ctas_per_sm(size_t smem) {
    // the occupancy of one architecture: the same on every device this library runs on
    static std::atomic<int> cached{0};
    int c = cached.load(std::memory_order_relaxed);
    if (c == 0) {
        int k = 0;
        if (cudaFuncSetAttribute(trsv_blocks<T, true, 1, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, trsv_blocks<T, true, 1, INV>, 32 * kTWarps, smem) !=
                cudaSuccess) {
            cudaGetLastError();
            k = 1;
        }
        c = std::max(1, k);
        cached.store(c, std::memory_order_relaxed);
    }
    return c;
}

template <typename T, bool INV>
static cudaError_t launch_trsv_per(int per, int grid, size_t smem, const T *LU, int lda, int n, int nq, T *X, int ldx,
                                   int *ws, int *status, long long bound_ns, cudaStream_t s, const T *Dinv) {
    switch (per) {
        case 1: return launch_trsv_nq<T, 1, INV>(grid, smem, LU, lda, n, nq, X, ldx, ws, status, bound_ns, s, Dinv);
        case 2: return launch_trsv_nq<T, 2, INV>(grid, smem, LU, lda, n, nq, X, ldx, ws, status, bound_ns, s, Dinv);
        case 4: return launch_trsv_nq<T, 4, INV>(grid, smem, LU, lda, n, nq, X, ldx, ws, status, bound_ns, s, Dinv);
        default: return launch_trsv_nq<T, 8, INV>(grid, smem, LU, lda, n, nq, X, ldx, ws, status, bound_ns, s, Dinv);
    }
}

// Workspace: trsv_workspace_ints(n, nrhs) ints, zeroed here before each pass.
// Dinv (may be NULL): the diagonal blocks' inverses from launch_diag_inverse;
// given, each block's diagonal solve is a product with its inverse (off the
// substitution chain's serial steps; the rounding differs from substitution,
// so it serves the refinement's preconditioner solves, not lu_solve).
template <typename T>
cudaError_t launch_trsv_pair(const T *LU, int lda, int n, int nrhs, T *X, int ldx, int *ws, int *status,
                             long long bound_ns, int sms, cudaStream_t s, const T *Dinv) {
    if (n <= 0 || nrhs <= 0) return cudaSuccess;
    const int nblk = (n + kTB - 1) / kTB;
    const size_t smem = sizeof(T) * (size_t)kTWarps * 2 * kTB * kTB;
    cudaError_t e = cudaSuccess;
    for (int q0 = 0; q0 < nrhs; q0 += kMaxRhs) {
        const int nq = std::min(kMaxRhs, nrhs - q0);
        // As many chains as keep every block's warp resident from the start (a block
        // whose warp starts late sums all its dependencies on the chain's critical
        // path), each carrying the fewest right-hand sides that allows.
        const int per_sm = Dinv ? trsv_ctas_per_sm<T, true>(smem) : trsv_ctas_per_sm<T, false>(smem);
        const int resident = std::max(1, per_sm) * kTWarps * sms;
        int chains = std::max(1, std::min(nq, resident / std::max(nblk, 1)));
        int per = (nq + chains - 1) / chains;
        per = per <= 1 ? 1 : per <= 2 ? 2 : per <= 4 ? 4 : 8;
        chains = (nq + per - 1) / per;
        const int grid = std::min((nblk * chains + kTWarps - 1) / kTWarps, 8 * sms);
        // tickets and the words of this pass's right-hand sides
        const size_t used = (size_t)2 * kFlagPad + (size_t)2 * TagWords<T>::value * nq * n;
        e = cudaMemsetAsync(ws, 0, sizeof(int) * used, s);
        if (e != cudaSuccess) return e;
        T *Xq = X + (size_t)q0 * ldx;
        if (Dinv) e = launch_trsv_per<T, true>(per, grid, smem, LU, lda, n, nq, Xq, ldx, ws, status, bound_ns, s, Dinv);
        else e = launch_trsv_per<T, false>(per, grid, smem, LU, lda, n, nq, Xq, ldx, ws, status, bound_ns, s, Dinv);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Self-test of the bounded waits: the forward substitution of an n x n unit
// lower triangle with the ticket of block 0 already taken, so no warp ever
// solves block 0 and every other block's poll of its words runs out after
// bound_ns.  The kernel then records LU_ERR_TIMEOUT in *status and returns;
// nothing faults and the context stays usable.  ws: trsv_workspace_ints(n, 1)
// ints; LU and X: n x n and n elements of FP32.
cudaError_t launch_trsv_timeout_selftest(const float *LU, int n, float *X, int *ws, int *status, long long bound_ns,
                                         cudaStream_t s) {
    if (n <= kTB) return cudaErrorInvalidValue;   // needs a second block to wait
    const size_t used = (size_t)2 * kFlagPad + (size_t)2 * TagWords<float>::value * n;
    cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(int) * used, s);
    if (e != cudaSuccess) return e;
    const int one = 1;
    e = cudaMemcpyAsync(ws, &one, sizeof(int), cudaMemcpyHostToDevice, s);   // block 0's ticket is gone
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float) * (size_t)kTWarps * 2 * kTB * kTB;
    e = cudaFuncSetAttribute(trsv_blocks<float, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nblk = (n + kTB - 1) / kTB;
    trsv_blocks<float, true, 1><<<(nblk + kTWarps - 1) / kTWarps, 32 * kTWarps, smem, s>>>(
        LU, n, n, 1, 1, X, n, ws, reinterpret_cast<unsigned long long *>(ws + 2 * kFlagPad), 1u, status, bound_ns);
    lu_count_launch();
    return cudaGetLastError();
}

// Self-test of lu_div_fast against the IEEE division: count mismatching bit
// patterns over the pairs in its safe range among `count` pairs drawn from a
// counter hash (both signs, every exponent, significands near 2 included).
template <typename T>
__global__ void div_selftest_kernel(long long count, unsigned long long seed, unsigned long long *mismatch) {
    unsigned long long bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        unsigned long long w = z * 0x9E3779B97F4A7C15ULL;
        w = (w ^ (w >> 30)) * 0xBF58476D1CE4E5B9ULL;
        w ^= w >> 27;
        T x, d;
        if constexpr (sizeof(T) == 4) {
            unsigned bx = (unsigned)z, bd = (unsigned)w;
            if ((i & 7) == 0) bd = (bd & 0x807fffffu) | (((bd >> 23) & 0xffu) << 23) | 0x007ffff0u;   // near-2 significands
            x = __uint_as_float(bx);
            d = __uint_as_float(bd);
        } else {
            unsigned long long bd = w;
            if ((i & 7) == 0) bd |= 0x000fffffffffff00ULL;
            x = __longlong_as_double((long long)z);
            d = __longlong_as_double((long long)bd);
        }
        if (x != x || d != d || d == T(0)) continue;
        if (!lu_div_safe(x, lu_div_range<T>::in(d))) continue;   // those take the IEEE division
        const T rcp = T(1) / d;
        const T a = lu_div_fast(x, d, rcp);
        const T b = x / d;
        bool same;
        if constexpr (sizeof(T) == 4) same = (__float_as_uint(a) == __float_as_uint(b)) || (a != a && b != b);
        else same = (__double_as_longlong(a) == __double_as_longlong(b)) || (a != a && b != b);
        if (!same) ++bad;
    }
    if (bad) atomicAdd(mismatch, bad);
}

cudaError_t launch_div_selftest(int dt64, long long count, unsigned long long seed, unsigned long long *mismatch,
                                cudaStream_t s) {
    if (dt64) div_selftest_kernel<double><<<1216, 256, 0, s>>>(count, seed, mismatch);
    else div_selftest_kernel<float><<<1216, 256, 0, s>>>(count, seed, mismatch);
    lu_count_launch();
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


template cudaError_t launch_gather_rows<double, double>(int, int, const int *, const double *, int, double *, int, cudaStream_t);
template cudaError_t launch_gather_rows<float, float>(int, int, const int *, const float *, int, float *, int, cudaStream_t);
template cudaError_t launch_trsv_pair<double>(const double *, int, int, int, double *, int, int *, int *, long long, int,
                                              cudaStream_t, const double *);
template cudaError_t launch_trsv_pair<float>(const float *, int, int, int, float *, int, int *, int *, long long, int,
                                             cudaStream_t, const float *);
template cudaError_t launch_diag_inverse<float>(const float *, int, int, float *, cudaStream_t);
template cudaError_t launch_diag_inverse<double>(const double *, int, int, double *, cudaStream_t);
template size_t trsv_inverse_elems<float>(int);
template size_t trsv_inverse_elems<double>(int);

}  // namespace lu
