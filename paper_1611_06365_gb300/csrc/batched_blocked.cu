// Batched LU with partial pivoting for orders up to 256: one persistent
// launch, CTAs taking matrices from a queue ordered largest first.
//
// Each matrix is factored by the blocked right-looking algorithm of section
// 3.1 (Figure 1, right) with panels of NB columns:
//   1. panel: thread i keeps row k+i of the panel in registers; per column a
//      block-wide (|a|, row) argmax (integer keys, warp reductions, one CTA
//      barrier), the interchange of the two rows' panel entries, IEEE
//      division and the rank-1 update inside the panel (section 3.1, RL1);
//   2. the panel's interchanges on all other columns, one column per thread
//      in LAPACK's order (laswp);
//   3. U12 := trilu(L11)^{-1} A12 by forward substitution: a warp takes
//      four columns at a time, lane r holding row r, and step q broadcasts
//      the finished x[q] with a shuffle (RL2);
//   4. A22 -= L21 U12, every element taking its NB updates in increasing
//      order (RL3).
// Every element thus sees exactly the fused multiply-adds, in the same order,
// of the unblocked algorithm with FMA, so the factors equal those of
// lu::getrf_batched_kernel bit for bit; the blocking only changes where the
// operands live (registers and shared memory instead of a full sweep of the
// matrix per column).  The matrices stay in global memory; each CTA works on
// one at a time, so its working set (at most 512 KiB) stays in L2.
#include "common.cuh"
#include "internal.h"
#include <algorithm>
#include <climits>

namespace lu {

constexpr int kBBThreads = 256;
constexpr int kBBWarps = kBBThreads / 32;
constexpr int kBBMaxN = 256;

template <typename T> struct BBVec;
template <> struct BBVec<float> { using type = float4; };
template <> struct BBVec<double> { using type = double2; };

template <typename T, int NB>
struct BBShared {
    static constexpr int VEC = 16 / sizeof(T);
    static constexpr int LS = NB + VEC;                  // row stride of L21 / U12 (16-byte aligned rows)
    __align__(16) T L21[kBBMaxN][LS];                    // the panel's rows (L11 on top), row-major
    __align__(16) T U12[kBBMaxN][LS];                    // column c of U12: its NB entries
    __align__(16) T wst[2][kBBWarps][NB];                // each warp's candidate row (double-buffered)
    __align__(16) T jst[2][NB];                          // row j of the panel
    unsigned long long red_key[2][kBBWarps];
    int red_idx[2][kBBWarps];
    int piv[NB];                                         // panel-local pivot rows
    int item;
};

__device__ __forceinline__ bool bb_key(float x, unsigned long long &k) {
    const unsigned b = __float_as_uint(x) & 0x7fffffffu;
    k = b;
    return b <= 0x7f800000u;   // NaN is never a candidate
}
__device__ __forceinline__ bool bb_key(double x, unsigned long long &k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    k = b;
    return b <= 0x7ff0000000000000ULL;
}
__device__ __forceinline__ bool bb_better(unsigned long long ka, int ia, unsigned long long kb, int ib) {
    return ka > kb || (ka == kb && ia < ib);
}
// warp-wide (key, row) maximum, smallest row on ties
__device__ __forceinline__ void bb_warp_argmax(unsigned long long &key, int &idx) {
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    const unsigned mine = (hi == mh && lo == ml) ? (unsigned)idx : 0xffffffffu;
    idx = (int)__reduce_min_sync(0xffffffffu, mine);
    key = ((unsigned long long)mh << 32) | ml;
}

__device__ __forceinline__ void bb_warp_argmax32(unsigned long long &key, int &idx) {
    const unsigned k32 = (unsigned)key;
    const unsigned mk = __reduce_max_sync(0xffffffffu, k32);
    idx = (int)__reduce_min_sync(0xffffffffu, k32 == mk ? (unsigned)idx : 0xffffffffu);
    key = mk;
}
template <typename T>
__device__ __forceinline__ void bb_argmax_t(unsigned long long &key, int &idx) {
    if constexpr (sizeof(T) == 4) bb_warp_argmax32(key, idx);
    else bb_warp_argmax(key, idx);
}

// Column step LJ of the panel on this thread's row i (panel-local): scaling
// and rank-1 update for i > LJ, and the candidate key of column LJ+1.
template <typename T, int NB, int LJ>
__device__ __forceinline__ void bb_rank1(T (&a)[NB], const T *__restrict__ urow, T pv, bool zero, int i, bool own, int w,
                                         unsigned long long &best, int &bidx) {
    using V = typename BBVec<T>::type;
    constexpr int VEC = 16 / sizeof(T);
    const bool act = own && i > LJ && !zero;
    if (act) {
        const T l = a[LJ] / pv;
        a[LJ] = l;
#pragma unroll
        for (int q = (LJ + 1) / VEC; q < NB / VEC; ++q) {
            V vv = reinterpret_cast<const V *>(urow)[q];
            const T *u = reinterpret_cast<const T *>(&vv);
#pragma unroll
            for (int v = 0; v < VEC; ++v)
                if (q * VEC + v > LJ) a[q * VEC + v] = fma(-l, u[v], a[q * VEC + v]);
        }
    }
    best = 0;
    bidx = INT_MAX;
    if constexpr (LJ + 1 < NB) {
        unsigned long long k;
        if (own && i > LJ && LJ + 1 < w && bb_key(a[LJ + 1], k)) { best = k; bidx = i; }
    }
}

#define LU_BB_CASE(L)                                                                                   \
    case (L):                                                                                           \
        if constexpr ((L) < NB) bb_rank1<T, NB, ((L) < NB ? (L) : 0)>(a, urow, pv, zero, tid, own, w, best, bidx); \
        break;
#define LU_BB_CASE4(L) LU_BB_CASE(L) LU_BB_CASE((L) + 1) LU_BB_CASE((L) + 2) LU_BB_CASE((L) + 3)
#define LU_BB_CASE16(L) LU_BB_CASE4(L) LU_BB_CASE4((L) + 4) LU_BB_CASE4((L) + 8) LU_BB_CASE4((L) + 12)

// Factor the n x n matrix A (n <= 256) in place; returns LAPACK's info.
template <typename T, int NB>
__device__ int bb_factor(BBShared<T, NB> &S, T *__restrict__ A, int lda, int n, int *__restrict__ ipiv) {
    using V = typename BBVec<T>::type;
    constexpr int VEC = 16 / sizeof(T);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int info = 0;
    unsigned colstep = 0;
    for (int k = 0; k < n; k += NB) {
        const int w = min(NB, n - k), m = n - k;
        const bool own = tid < m;
        // ---- 1. panel -------------------------------------------------------------
        T a[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) a[c] = (own && c < w) ? A[(size_t)(k + tid) + (size_t)(k + c) * lda] : T(0);
        unsigned long long best = 0;
        int bidx = INT_MAX;
        {
            unsigned long long kk;
            if (own && bb_key(a[0], kk)) { best = kk; bidx = tid; }
        }
        for (int lj = 0; lj < w; ++lj) {
            const int par = colstep & 1;
            ++colstep;
            bb_argmax_t<T>(best, bidx);
            if (bidx != INT_MAX && lane == (bidx & 31)) {
#pragma unroll
                for (int q = 0; q < NB / VEC; ++q) reinterpret_cast<V *>(S.wst[par][warp])[q] = reinterpret_cast<const V *>(a)[q];
            }
            if (tid == lj) {
#pragma unroll
                for (int q = 0; q < NB / VEC; ++q) reinterpret_cast<V *>(S.jst[par])[q] = reinterpret_cast<const V *>(a)[q];
            }
            if (lane == 0) { S.red_key[par][warp] = best; S.red_idx[par][warp] = bidx; }
            __syncthreads();
            unsigned long long ck = lane < kBBWarps ? S.red_key[par][lane] : 0ULL;
            int cr = lane < kBBWarps ? S.red_idx[par][lane] : INT_MAX;
            bb_argmax_t<T>(ck, cr);
            const bool valid = cr != INT_MAX;
            const int p = valid ? cr : lj;   // no candidate (all NaN): keep row lj
            const T *urow = valid ? S.wst[par][cr >> 5] : S.jst[par];
            const T *drow = S.jst[par];
            const T pv = urow[lj];
            const bool zero = (pv == T(0));
            if (tid == 0) S.piv[lj] = zero ? lj : p;
            if (zero && info == 0) info = k + lj + 1;
            if (!zero && p != lj && (tid == lj || tid == p)) {
                const T *src = tid == lj ? urow : drow;
#pragma unroll
                for (int q = 0; q < NB / VEC; ++q) reinterpret_cast<V *>(a)[q] = reinterpret_cast<const V *>(src)[q];
            }
            switch (lj) {
                LU_BB_CASE16(0)
                LU_BB_CASE16(16)
                default: break;
            }
        }
        // panel back to memory; its rows to shared memory for the solve and the update
        if (own) {
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c < w) A[(size_t)(k + tid) + (size_t)(k + c) * lda] = a[c];
#pragma unroll
            for (int q = 0; q < NB / VEC; ++q) reinterpret_cast<V *>(S.L21[tid])[q] = reinterpret_cast<const V *>(a)[q];
        }
        __syncthreads();
        if (tid < w) ipiv[k + tid] = k + S.piv[tid] + 1;
        // ---- 2. interchanges on the other columns, in order ------------------------
        {
            const int nother = n - w;   // columns [0, k) and [k + w, n)
            for (int cc = tid; cc < nother; cc += kBBThreads) {
                T *colp = A + (size_t)(cc < k ? cc : cc + w) * lda + k;
                // bring the column's rows k..n-1 into L1 first: the interchanges
                // below are a dependent chain of loads and stores
                for (int r = 0; r < m; r += 128 / (int)sizeof(T))
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(colp + r));
                for (int j = 0; j < w; ++j) {
                    const int q = S.piv[j];
                    if (q != j) {
                        const T t0 = colp[j], t1 = colp[q];
                        colp[j] = t1;
                        colp[q] = t0;
                    }
                }
            }
        }
        __syncthreads();
        // ---- 3. U12 := trilu(L11)^{-1} A12 ------------------------------------------
        const int nc = n - k - w;
        if (nc == 0) break;   // last panel: nothing to its right
        {
            const int r = lane;   // row of the block
            T lrow[NB];
#pragma unroll
            for (int q = 0; q < NB / VEC; ++q) reinterpret_cast<V *>(lrow)[q] = reinterpret_cast<const V *>(S.L21[r < w ? r : 0])[q];
            constexpr int TC = 4;   // columns per warp pass
            for (int cb = warp * TC; cb < nc; cb += kBBWarps * TC) {
                T x[TC];
#pragma unroll
                for (int u = 0; u < TC; ++u)
                    x[u] = (r < w && cb + u < nc) ? A[(size_t)(k + r) + (size_t)(k + w + cb + u) * lda] : T(0);
#pragma unroll
                for (int q = 0; q < NB - 1; ++q) {
                    if (q + 1 < w) {
#pragma unroll
                        for (int u = 0; u < TC; ++u) {
                            const T xq = __shfl_sync(0xffffffffu, x[u], q);
                            if (r > q) x[u] = fma(-lrow[q], xq, x[u]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < TC; ++u) {
                    if (cb + u < nc) {
                        if (r < w) A[(size_t)(k + r) + (size_t)(k + w + cb + u) * lda] = x[u];
                        if (r < NB) S.U12[cb + u][r] = r < w ? x[u] : T(0);
                    }
                }
            }
        }
        __syncthreads();
        // ---- 4. A22 -= L21 U12 ------------------------------------------------------
        {
            const int R = m - w;                        // rows below the panel's top block
            const int RP = (R + 31) & ~31;              // whole warps per row set
            const int G = max(1, kBBThreads / RP);      // column groups
            const int r = tid % RP, g = tid / RP;
            if (r < R && g < G) {
                T l[NB];
#pragma unroll
                for (int q = 0; q < NB / VEC; ++q) reinterpret_cast<V *>(l)[q] = reinterpret_cast<const V *>(S.L21[w + r])[q];
                T *rowp = A + (size_t)(k + w + r) + (size_t)(k + w) * lda;
                // four columns (c, c+G, c+2G, c+3G) per step; the next four are
                // loaded before this step's products (software pipelining)
                constexpr int CG = 4;
                T xc[CG], xn[CG];
#pragma unroll
                for (int v = 0; v < CG; ++v) xc[v] = g + v * G < nc ? rowp[(size_t)(g + v * G) * lda] : T(0);
                for (int c = g; c < nc; c += CG * G) {
#pragma unroll
                    for (int v = 0; v < CG; ++v) {
                        const int cn = c + (CG + v) * G;
                        xn[v] = cn < nc ? rowp[(size_t)cn * lda] : T(0);
                    }
#pragma unroll
                    for (int q = 0; q < NB / VEC; ++q) {
#pragma unroll
                        for (int v = 0; v < CG; ++v) {
                            const int cv = c + v * G;
                            V uv = reinterpret_cast<const V *>(S.U12[cv < nc ? cv : 0])[q];
                            const T *up = reinterpret_cast<const T *>(&uv);
#pragma unroll
                            for (int e = 0; e < VEC; ++e)
                                if (q * VEC + e < w) xc[v] = fma(-l[q * VEC + e], up[e], xc[v]);
                        }
                    }
#pragma unroll
                    for (int v = 0; v < CG; ++v) {
                        const int cv = c + v * G;
                        if (cv < nc) rowp[(size_t)cv * lda] = xc[v];
                        xc[v] = xn[v];
                    }
                }
            }
        }
        __syncthreads();
    }
    return info;
}

// two CTAs per SM; three for FP32 with 16-column panels (fewer registers and
// less shared memory), so more matrices are in flight to hide L2 latency
template <typename T, int NB>
__global__ void __launch_bounds__(kBBThreads, (sizeof(T) == 4 && NB == 16) ? 3 : 2)
getrf_batched_blocked(const int *__restrict__ ns, T *const *__restrict__ As, const int *__restrict__ ldas,
                      int *const *__restrict__ ipivs, int *__restrict__ infos, const int *__restrict__ order, int count,
                      int *__restrict__ queue) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BBShared<T, NB> &S = *reinterpret_cast<BBShared<T, NB> *>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) S.item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = S.item;
        __syncthreads();
        if (it >= count) break;
        const int t = order[it];
        const int n = ns[t];
        const int info = n > 0 ? bb_factor<T, NB>(S, As[t], ldas[t], n, ipivs[t]) : 0;
        if (threadIdx.x == 0) infos[t] = info;
    }
}

// order[] = the batch indices sorted by order n, largest first (counting
// sort over n in [0, kBBMaxN]); also clears the queue counter.  One CTA.
__global__ void __launch_bounds__(1024) bb_order_kernel(const int *__restrict__ ns, int count, int *__restrict__ order,
                                                       int *__restrict__ queue) {
    __shared__ int hist[kBBMaxN + 1], start[kBBMaxN + 1];
    for (int i = threadIdx.x; i <= kBBMaxN; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < count; t += blockDim.x) atomicAdd(&hist[kBBMaxN - min(max(ns[t], 0), kBBMaxN)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int i = 0; i <= kBBMaxN; ++i) { start[i] = s; s += hist[i]; }
        *queue = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < count; t += blockDim.x) {
        const int b = kBBMaxN - min(max(ns[t], 0), kBBMaxN);
        order[atomicAdd(&start[b], 1)] = t;
    }
}

// Batched solve for orders up to 256: one warp per (matrix, right-hand side).
// The interchanges are applied in order to b in shared memory; then both
// substitutions run by blocks of 32 rows, lane r holding row r of the block:
// the products of the finished blocks (columns of L or U read coalesced, the
// finished x broadcast by shuffles) and the 32-step solve of the diagonal
// block, in the same order of operations for every element as the plain
// column-oriented substitution.
template <typename T>
__global__ void __launch_bounds__(256)
getrs_batched_warp(int batch, int nrhs, const int *__restrict__ ns, const T *const *__restrict__ LUs,
                   const int *__restrict__ ldas, const int *const *__restrict__ ipivs, T *const *__restrict__ Bs,
                   const int *__restrict__ ldbs) {
    __shared__ __align__(16) T xs_all[8][kBBMaxN];
    __shared__ int pv_all[8][kBBMaxN];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    T *xs = xs_all[wib];
    int *pv = pv_all[wib];
    const long long nwork = (long long)batch * nrhs;
    for (long long wk = (long long)blockIdx.x * 8 + wib; wk < nwork; wk += (long long)gridDim.x * 8) {
        const int t = (int)(wk / nrhs), q = (int)(wk % nrhs);
        const int n = ns[t], lda = ldas[t];
        if (n <= 0) continue;
        const T *LU = LUs[t];
        const int *ipiv = ipivs[t];
        T *b = Bs[t] + (size_t)q * ldbs[t];
        for (int i = lane; i < n; i += 32) {
            xs[i] = b[i];
            pv[i] = ipiv[i] - 1;
        }
        __syncwarp();
        if (lane == 0)
            for (int j = 0; j < n; ++j) {
                const int p = pv[j];
                if (p != j) { const T u = xs[j]; xs[j] = xs[p]; xs[p] = u; }
            }
        __syncwarp();
        using V = typename BBVec<T>::type;
        constexpr int VEC = 16 / sizeof(T);
        const int nblk = (n + 31) >> 5;
        // forward: unit lower; x lives in shared memory (finished blocks are read
        // back as broadcasts), each 32 x 32 tile is loaded whole before its products
        for (int I = 0; I < nblk; ++I) {
            const int r = I * 32 + lane;
            const bool has = r < n;
            T acc = has ? xs[r] : T(0);
            for (int J = 0; J <= I; ++J) {
                const int cols = min(32, n - J * 32);
                T l[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) l[c] = (has && c < cols) ? LU[(size_t)r + (size_t)(J * 32 + c) * lda] : T(0);
                if (J < I) {
#pragma unroll
                    for (int c4 = 0; c4 < 32 / VEC; ++c4) {
                        V xv = reinterpret_cast<const V *>(xs + J * 32)[c4];
                        const T *xp = reinterpret_cast<const T *>(&xv);
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            if (c4 * VEC + v < cols) acc = fma(-l[c4 * VEC + v], xp[v], acc);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 31; ++c) {
                        const T xc = __shfl_sync(0xffffffffu, acc, c);
                        if (lane > c && c < cols) acc = fma(-l[c], xc, acc);
                    }
                }
            }
            if (has) xs[r] = acc;
            __syncwarp();
        }
        // backward: upper, columns in decreasing order
        for (int I = nblk - 1; I >= 0; --I) {
            const int r = I * 32 + lane;
            const bool has = r < n;
            T acc = has ? xs[r] : T(0);
            for (int J = nblk - 1; J >= I; --J) {
                const int cols = min(32, n - J * 32);
                T u[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) u[c] = (has && c < cols) ? LU[(size_t)r + (size_t)(J * 32 + c) * lda] : T(0);
                if (J > I) {
#pragma unroll
                    for (int c4 = 32 / VEC - 1; c4 >= 0; --c4) {
                        V xv = reinterpret_cast<const V *>(xs + J * 32)[c4];
                        const T *xp = reinterpret_cast<const T *>(&xv);
#pragma unroll
                        for (int v = VEC - 1; v >= 0; --v)   // entries past n of a short last block are not data
                            if (c4 * VEC + v < cols) acc = fma(-u[c4 * VEC + v], xp[v], acc);
                    }
                } else {
                    // diagonal block: lane c holds u(r, r) in u[lane]; its reciprocal off the
                    // chain, lu_div_fast on the chain, the IEEE division again if any lane's
                    // division left the safe range
                    T dg = u[0];
#pragma unroll
                    for (int c = 1; c < 32; ++c)
                        if (lane == c) dg = u[c];
                    if (!has) dg = T(1);
                    const T rdg = T(1) / dg;
                    const bool okd = lu_div_range<T>::in(dg);
                    const T acc0 = acc;
                    T pre = T(0);   // the operand of this lane's division, checked after the chain
#pragma unroll
                    for (int c = 31; c >= 0; --c) {
                        if (c < cols) {
                            if (lane == c) {
                                pre = acc;
                                acc = lu_div_fast(acc, dg, rdg);
                            }
                            const T xc = __shfl_sync(0xffffffffu, acc, c);
                            if (lane < c) acc = fma(-u[c], xc, acc);
                        }
                    }
                    if (__any_sync(0xffffffffu, has && !lu_div_safe(pre, okd))) {
                        acc = acc0;
#pragma unroll
                        for (int c = 31; c >= 0; --c) {
                            if (c < cols) {
                                if (lane == c) acc = acc / dg;
                                const T xc = __shfl_sync(0xffffffffu, acc, c);
                                if (lane < c) acc = fma(-u[c], xc, acc);
                            }
                        }
                    }
                }
            }
            if (has) xs[r] = acc;
            __syncwarp();
        }
        for (int i = lane; i < n; i += 32) b[i] = xs[i];
        __syncwarp();
    }
}

template <typename T>
cudaError_t launch_getrs_batched_warp(int batch, int nrhs, const int *ns, const T *const *LUs, const int *ldas,
                                      const int *const *ipivs, T *const *Bs, const int *ldbs, int sms, cudaStream_t s) {
    if (batch <= 0 || nrhs <= 0) return cudaSuccess;
    const long long work = (long long)batch * nrhs;
    const int grid = (int)std::min<long long>((work + 7) / 8, (long long)sms * 8);
    getrs_batched_warp<T><<<grid, 256, 0, s>>>(batch, nrhs, ns, LUs, ldas, ipivs, Bs, ldbs);
    lu_count_launch();
    return cudaGetLastError();
}

size_t batched_blocked_workspace_ints(int batch) { return (size_t)batch + 32; }

template <typename T, int NB>
static cudaError_t launch_bb(int batch, const int *ns, T *const *As, const int *ldas, int *const *ipivs, int *infos,
                             int *ws, int sms, cudaStream_t s) {
    const size_t smem = sizeof(BBShared<T, NB>);
    cudaError_t e = cudaFuncSetAttribute(getrf_batched_blocked<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, getrf_batched_blocked<T, NB>, kBBThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, per_sm);
    int *queue = ws, *order = ws + 32;
    bb_order_kernel<<<1, 1024, 0, s>>>(ns, batch, order, queue);
    lu_count_launch();
    const int grid = std::min(batch, sms * per_sm);
    getrf_batched_blocked<T, NB><<<grid, kBBThreads, smem, s>>>(ns, As, ldas, ipivs, infos, order, batch, queue);
    lu_count_launch();
    return cudaGetLastError();
}

// Blocked batched factorization for max_n <= 256; nb = panel width (16 or
// 32; 0 picks 16: the panel's per-column chain is the latency that matters).  ws: batched_blocked_workspace_ints
// ints of device memory.
template <typename T>
cudaError_t launch_getrf_batched_blocked(int batch, const int *ns, T *const *As, const int *ldas, int *const *ipivs,
                                         int *infos, int nb, int *ws, int sms, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    if (nb == 0) nb = 16;
    if (nb == 32) return launch_bb<T, 32>(batch, ns, As, ldas, ipivs, infos, ws, sms, s);
    if (nb == 16) return launch_bb<T, 16>(batch, ns, As, ldas, ipivs, infos, ws, sms, s);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_getrs_batched_warp<double>(int, int, const int *, const double *const *, const int *,
                                                       const int *const *, double *const *, const int *, int, cudaStream_t);
template cudaError_t launch_getrs_batched_warp<float>(int, int, const int *, const float *const *, const int *,
                                                      const int *const *, float *const *, const int *, int, cudaStream_t);
template cudaError_t launch_getrf_batched_blocked<double>(int, const int *, double *const *, const int *, int *const *, int *,
                                                          int, int *, int, cudaStream_t);
template cudaError_t launch_getrf_batched_blocked<float>(int, const int *, float *const *, const int *, int *const *, int *,
                                                         int, int *, int, cudaStream_t);

}  // namespace lu
