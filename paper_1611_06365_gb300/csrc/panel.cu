// Panel factorization (RL1 / PF3 of the paper) on one thread-block cluster.
//
// One launch factors a whole outer panel of b_o columns (section 3.1,
// Figure 1; the outer/inner split of section 4.2, Figure 6).  The panel's m
// rows are split over the C <= 16 CTAs of a cluster (R rows each).  The inner
// panel of b_i columns lives in shared memory; per column j:
//
//   1. every CTA reduces the (|a|, row) maximum of its rows (warp shuffles,
//      then shared memory), and PUSHES the candidate (magnitude, row, the
//      row's b_i values) into a slot of every CTA of the cluster with
//      distributed-shared-memory stores; the CTA holding row j pushes row j;
//   2. one hardware cluster barrier (release/acquire) per column;
//   3. every CTA picks the winner locally (largest magnitude, smallest row on
//      ties) and the two owners write the interchanged rows;
//   4. every CTA scales its part of column j by IEEE division and applies the
//      rank-1 update to its rows, tracking the candidate of column j+1.
//
// After each inner panel (when b_o > b_i), still inside the same launch:
// its interchanges are applied to the panel's other columns (one row map,
// gather then scatter), U12 := trilu(L11)^{-1} A12 is formed, and the inner
// trailing update A22 -= L21 U12 runs on each CTA's own rows.  At the end the
// kernel builds the row map of all b_o interchanges for the rest of the
// matrix, updates the permutation vector, and, for the tensor-core update,
// stages L21 as BF16 (optionally split hi/lo) in K-major order.
//
// Candidate and row-j slots are double-buffered by column parity, so one
// cluster barrier per column suffices: a CTA writes slot (j+2) & 1 of a peer
// only after passing barrier j+1, which the peer reaches after reading slot
// j & 1.
#include "common.cuh"
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <climits>

namespace cg = cooperative_groups;

namespace lu {

constexpr int kPanelThreads = 512;
constexpr int kPanelWMax = 64;       // inner panel width b_i
constexpr int kPanelBoMax = 256;     // outer panel width b_o
constexpr int kPanelMaxCtas = 16;
// end-of-panel scratch carved from As: row map (6 b_o ints) + probe table (2 x 4096 ints),
// or the BF16 staging tile (32 rows x b_o floats)
constexpr size_t kPanelScratch = sizeof(int) * (6 * kPanelBoMax + 8192);

template <typename T>
struct __align__(16) CandSlot {
    T mag;
    int row;
    int pad[(16 - sizeof(T) - sizeof(int)) / sizeof(int)];   // vals start 16-byte aligned
    T vals[kPanelWMax];
};

template <typename T>
struct PanelShared {
    CandSlot<T> cand[2][kPanelMaxCtas];   // pushed by every CTA (double-buffered)
    __align__(16) T diag[2][kPanelWMax];  // row j, pushed by its owner
    T urow[kPanelWMax], drow[kPanelWMax];
    T red_mag[32];
    int red_idx[32];
    int bc[4];
    int piv[kPanelBoMax];                 // this panel's pivots (panel-local rows)
    int map_rows[2 * kPanelWMax], map_src[2 * kPanelWMax];
    int map_cnt;
    int cnt_s;
    int first_zero;                       // first column with a zero pivot (-1: none)
};

template <typename T>
__device__ __forceinline__ void warp_argmax(T &mag, int &idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T m2 = __shfl_xor_sync(0xffffffffu, mag, o);
        int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (lu_better(m2, i2, mag, idx)) { mag = m2; idx = i2; }
    }
}

static inline size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }

// Dynamic shared memory: PanelShared | As[bi][R] (column-major) | U12s[bo-1][bi+1] | gv[ceil(bo/C)][2 bi] | L11s[bi][bi]
template <typename T>
struct PanelLayout {
    size_t as_off, u12_off, gv_off, l11_off, total;
    __host__ __device__ PanelLayout(int R, int bi, int bo, int C) {
        as_off = (sizeof(PanelShared<T>) + 15) & ~(size_t)15;
        u12_off = as_off + (((size_t)R * bi * sizeof(T) + 15) & ~(size_t)15);
        // an inner panel of width wi >= 1 leaves at most bo - 1 columns to its
        // right (A12) and bo - 1 other columns in all (a short inner panel, or a
        // panel with fewer rows than columns, leaves more than bo - bi)
        const int nright = bo > 1 ? bo - 1 : 0;
        gv_off = u12_off + (((size_t)(bi + 1) * nright * sizeof(T) + 15) & ~(size_t)15);
        const int nother = bo > 1 ? bo : 0;
        const int ncols = C > 0 ? (nother + C - 1) / C : nother;
        l11_off = gv_off + (((size_t)2 * bi * ncols * sizeof(T) + 15) & ~(size_t)15);
        total = l11_off + (bo > bi ? (size_t)bi * bi * sizeof(T) : 0) + 16;
    }
};

// Row map of the sequential interchanges p[0..cnt) of rows r0.. (panel-local):
// rows[s] receives the old content of src[s].  One thread.
__device__ int make_row_map(const int *p, int r0, int cnt, int *rows, int *src) {
    int n = cnt;
    for (int t = 0; t < cnt; ++t) { rows[t] = r0 + t; src[t] = r0 + t; }
    for (int j = 0; j < cnt; ++j) {
        const int q = p[j];
        if (q == r0 + j) continue;
        int iq = -1;
        if (q < r0 + cnt) {
            iq = q - r0;
        } else {
            for (int s = cnt; s < n; ++s)
                if (rows[s] == q) { iq = s; break; }
            if (iq < 0) { rows[n] = q; src[n] = q; iq = n++; }
        }
        const int tmp = src[j];
        src[j] = src[iq];
        src[iq] = tmp;
    }
    return n;
}

template <typename T>
__global__ void __launch_bounds__(kPanelThreads, 1)
panel_factor_cluster(T *__restrict__ P, int lda, int m, int bo, int bi, int R, int *__restrict__ ipiv, int row_base,
                     int *__restrict__ info, int *__restrict__ map_out, int *__restrict__ perm,
                     __nv_bfloat16 *__restrict__ stage, int lds, int kpad, int split) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kPanelThreads / 32;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PanelLayout<T> lay(R, bi, bo, C);
    PanelShared<T> &S = *reinterpret_cast<PanelShared<T> *>(smem_raw);
    T *As = reinterpret_cast<T *>(smem_raw + lay.as_off);
    T *U12s = reinterpret_cast<T *>(smem_raw + lay.u12_off);
    T *gv = reinterpret_cast<T *>(smem_raw + lay.gv_off);
    T *L11s = reinterpret_cast<T *>(smem_raw + lay.l11_off);   // [wi][wi] column-major, inner transitions

    const int r0 = rank * R;
    const int myR = max(0, min(R, m - r0));
    const int kmax = min(m, bo);
    if (tid == 0) S.first_zero = -1;

    for (int jb = 0; jb < kmax; jb += bi) {
        const int wi = min(bi, kmax - jb);
        // (a) own rows of the inner columns into shared memory
        for (int c = 0; c < wi; ++c)
            for (int lr = tid; lr < myR; lr += kPanelThreads)
                As[(size_t)c * R + lr] = P[(size_t)(r0 + lr) + (size_t)(jb + c) * lda];
        __syncthreads();
        T best = T(-1);
        int bidx = INT_MAX;
        for (int lr = tid; lr < myR; lr += kPanelThreads) {
            const int i = r0 + lr;
            if (i < jb) continue;
            T v = lu_abs(As[lr]);
            if (lu_better(v, i, best, bidx)) { best = v; bidx = i; }
        }
        // (b) column steps: one CTA barrier and one cluster barrier per column
        constexpr int VEC = 16 / sizeof(T);          // values per 16-byte DSMEM store
        for (int lj = 0; lj < wi; ++lj) {
            const int j = jb + lj;
            const int par = j & 1;
            warp_argmax(best, bidx);
            if (lane == 0) { S.red_mag[warp] = best; S.red_idx[warp] = bidx; }
            __syncthreads();   // also orders the previous step's updates before the reads below
            // every warp reduces the warp candidates itself (no second barrier)
            T cmag = lane < nwarps ? S.red_mag[lane] : T(-1);
            int crow = lane < nwarps ? S.red_idx[lane] : INT_MAX;
            warp_argmax(cmag, crow);
            const bool own_j = (j >= r0 && j < r0 + myR);
            // push the candidate (and row j) into every CTA's slots, 16 bytes per store
            const int nvec = (wi + VEC - 1) / VEC;
            for (int e = tid; e < C * (nvec + 1); e += kPanelThreads) {
                const int d = e / (nvec + 1), q = e % (nvec + 1);
                CandSlot<T> *dst = cl.map_shared_rank(&S.cand[par][rank], d);
                if (q == 0) {
                    dst->mag = cmag;
                    dst->row = crow;
                } else if (crow != INT_MAX) {
                    T v[VEC];
#pragma unroll
                    for (int u = 0; u < VEC; ++u) {
                        const int c = (q - 1) * VEC + u;
                        v[u] = c < wi ? As[(size_t)c * R + (crow - r0)] : T(0);
                    }
                    *reinterpret_cast<float4 *>(&dst->vals[(q - 1) * VEC]) = *reinterpret_cast<float4 *>(v);
                }
            }
            if (own_j)
                for (int e = tid; e < C * nvec; e += kPanelThreads) {
                    const int d = e / nvec, q = e % nvec;
                    T v[VEC];
#pragma unroll
                    for (int u = 0; u < VEC; ++u) {
                        const int c = q * VEC + u;
                        v[u] = c < wi ? As[(size_t)c * R + (j - r0)] : T(0);
                    }
                    T *dst = cl.map_shared_rank(&S.diag[par][0], d);
                    *reinterpret_cast<float4 *>(&dst[q * VEC]) = *reinterpret_cast<float4 *>(v);
                }
            cl.sync();
            // winner from the local copies, reduced by every warp (no barrier)
            T mg = lane < C ? S.cand[par][lane].mag : T(-1);
            int ix = lane < C ? S.cand[par][lane].row : INT_MAX;
            int src = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                T m2 = __shfl_xor_sync(0xffffffffu, mg, o);
                int i2 = __shfl_xor_sync(0xffffffffu, ix, o);
                int s2 = __shfl_xor_sync(0xffffffffu, src, o);
                if (lu_better(m2, i2, mg, ix)) { mg = m2; ix = i2; src = s2; }
            }
            const bool valid = (ix != INT_MAX);
            const int p = valid ? ix : j;   // every candidate NaN: keep row j, as a sequential scan would
            const T *urow = valid ? S.cand[par][src].vals : S.diag[par];
            const T *drow = S.diag[par];    // old row j, the new content of row p
            const T pv = urow[lj];
            const bool zero = (pv == T(0));
            const int pfinal = zero ? j : p;
            if (tid == 0) {
                S.piv[j] = pfinal;
                if (zero && S.first_zero < 0) S.first_zero = j;
            }
            // row j becomes the pivot row (nobody reads it again in this panel step)
            if (!zero && p != j && own_j && tid < wi) As[(size_t)tid * R + (j - r0)] = urow[tid];
            best = T(-1);
            bidx = INT_MAX;
            const bool has_next = (lj + 1 < wi);
            for (int lr = tid; lr < myR; lr += kPanelThreads) {
                const int i = r0 + lr;
                if (i <= j) continue;
                if (!zero) {
                    // row p takes the old row j before its own update
                    const bool swapped = (i == p && p != j);
                    if (swapped)   // the factored columns of row p are row j's as well
                        for (int c = 0; c < lj; ++c) As[(size_t)c * R + lr] = drow[c];
                    const T l = (swapped ? drow[lj] : As[(size_t)lj * R + lr]) / pv;
                    As[(size_t)lj * R + lr] = l;
                    for (int c = lj + 1; c < wi; ++c) {
                        T *a = &As[(size_t)c * R + lr];
                        *a = fma(-l, urow[c], swapped ? drow[c] : *a);
                    }
                }
                if (has_next) {
                    T v = lu_abs(As[(size_t)(lj + 1) * R + lr]);
                    if (lu_better(v, i, best, bidx)) { best = v; bidx = i; }
                }
            }
        }
        __syncthreads();
        // (c) the factored inner panel back to global memory
        for (int c = 0; c < wi; ++c)
            for (int lr = tid; lr < myR; lr += kPanelThreads)
                P[(size_t)(r0 + lr) + (size_t)(jb + c) * lda] = As[(size_t)c * R + lr];
        if (wi >= bo) break;   // the panel is a single inner panel
        cl.sync();
        // (d) the inner interchanges on the panel's other columns, split over the cluster by columns
        if (tid == 0) S.map_cnt = make_row_map(S.piv + jb, jb, wi, S.map_rows, S.map_src);
        __syncthreads();
        {
            const int cnt = S.map_cnt;
            const int nother = bo - wi;   // columns [0, jb) and [jb + wi, bo)
            const int per = (nother + C - 1) / C;
            const int c_lo = rank * per, c_hi = min(nother, c_lo + per);
            const int ncols = max(0, c_hi - c_lo);
            for (int e = tid; e < cnt * ncols; e += kPanelThreads) {
                const int s = e % cnt, cc = c_lo + e / cnt;
                const int col = cc < jb ? cc : cc + wi;
                gv[(size_t)(e / cnt) * (2 * bi) + s] = P[(size_t)S.map_src[s] + (size_t)col * lda];
            }
            __syncthreads();
            for (int e = tid; e < cnt * ncols; e += kPanelThreads) {
                const int s = e % cnt, cc = c_lo + e / cnt;
                const int col = cc < jb ? cc : cc + wi;
                P[(size_t)S.map_rows[s] + (size_t)col * lda] = gv[(size_t)(e / cnt) * (2 * bi) + s];
            }
        }
        cl.sync();
        const int c_right = jb + wi, nr = bo - c_right;
        if (nr > 0) {
            // (e) U12 := trilu(L11)^{-1} A12, formed by every CTA in shared memory
            for (int e = tid; e < wi * nr; e += kPanelThreads) {
                const int r = e % wi, c = e / wi;
                U12s[(size_t)c * (wi + 1) + r] = P[(size_t)(jb + r) + (size_t)(c_right + c) * lda];
            }
            for (int e = tid; e < wi * wi; e += kPanelThreads) {
                const int r = e % wi, c = e / wi;
                L11s[(size_t)c * wi + r] = P[(size_t)(jb + r) + (size_t)(jb + c) * lda];
            }
            cl.sync();   // every CTA holds A12 before CTA 0 overwrites it with U12
            for (int c = tid; c < nr; c += kPanelThreads) {
                T *x = &U12s[(size_t)c * (wi + 1)];   // odd stride: no bank conflicts across columns
                for (int kk = 0; kk < wi; ++kk) {
                    const T xk = x[kk];
                    for (int r = kk + 1; r < wi; ++r) x[r] = fma(-L11s[(size_t)kk * wi + r], xk, x[r]);
                }
            }
            __syncthreads();
            if (rank == 0)
                for (int e = tid; e < wi * nr; e += kPanelThreads) {
                    const int r = e % wi, c = e / wi;
                    P[(size_t)(jb + r) + (size_t)(c_right + c) * lda] = U12s[(size_t)c * (wi + 1) + r];
                }
            // (f) inner update of this CTA's rows below the inner panel: A22 -= L21 U12,
            // 4 rows x 4 columns per thread (rows r0 + lr, lr = rq + 32 * u)
            {
                const int lo = max(0, c_right - r0);          // first own row below the inner panel
                const int nrow = myR - lo;
                const int rgroups = (nrow + 127) / 128, cgroups = (nr + 3) / 4;
                for (int g = tid; g < rgroups * 32 * cgroups; g += kPanelThreads) {
                    const int rq = g % 32, rest = g / 32;
                    const int rb = rest % rgroups, cb = rest / rgroups;
                    const int lr0 = lo + rb * 128 + rq, c0 = cb * 4;
                    T acc[4][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
                    for (int kk = 0; kk < wi; ++kk) {
                        T a[4], bq[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int lr = lr0 + 32 * u;
                            a[u] = lr < myR ? As[(size_t)kk * R + lr] : T(0);
                        }
#pragma unroll
                        for (int v = 0; v < 4; ++v) bq[v] = c0 + v < nr ? U12s[(size_t)(c0 + v) * (wi + 1) + kk] : T(0);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bq[v], acc[u][v]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int lr = lr0 + 32 * u;
                        if (lr >= myR) continue;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            if (c0 + v >= nr) continue;
                            T *a = &P[(size_t)(r0 + lr) + (size_t)(c_right + c0 + v) * lda];
                            *a = *a - acc[u][v];
                        }
                    }
                }
            }
        }
        cl.sync();
    }
    cl.sync();   // all of the panel is final in global memory
    // pivots and the first zero pivot, written once per panel
    if (rank == 0) {
        for (int j = tid; j < kmax; j += kPanelThreads) ipiv[j] = row_base + S.piv[j] + 1;
        if (tid == 0 && S.first_zero >= 0) atomicCAS(info, 0, row_base + S.first_zero + 1);
    }

    // row map of all the panel's interchanges, for the rest of the matrix:
    // [0] count, [1 .. 1+2bo) rows, [1+2bo .. 1+4bo) src (matrix rows)
    if (rank == 0 && map_out) {
        int *rows = reinterpret_cast<int *>(As);
        int *src = rows + 2 * kPanelBoMax;
        int *old = src + 2 * kPanelBoMax;
        int *keys = old + 2 * kPanelBoMax;
        int *slot = keys + 4096;
        for (int i = tid; i < 4096; i += kPanelThreads) keys[i] = -1;
        __syncthreads();
        if (tid == 0) {
            int n = kmax;
            for (int t = 0; t < kmax; ++t) { rows[t] = t; src[t] = t; }
            for (int j = 0; j < kmax; ++j) {
                const int q = S.piv[j];
                if (q == j) continue;
                int iq;
                if (q < kmax) {
                    iq = q;
                } else {
                    unsigned h = ((unsigned)q * 2654435761u) & 4095u;
                    while (keys[h] != -1 && keys[h] != q) h = (h + 1) & 4095u;
                    if (keys[h] == -1) { keys[h] = q; slot[h] = n; rows[n] = q; src[n] = q; ++n; }
                    iq = slot[h];
                }
                const int tmp = src[j];
                src[j] = src[iq];
                src[iq] = tmp;
            }
            S.cnt_s = n;
            map_out[0] = n;
        }
        __syncthreads();
        const int n = S.cnt_s;
        for (int s = tid; s < n; s += kPanelThreads) {
            map_out[1 + s] = row_base + rows[s];
            map_out[1 + 2 * bo + s] = row_base + src[s];
        }
        if (perm) {
            for (int s = tid; s < n; s += kPanelThreads) old[s] = perm[row_base + src[s]];
            __syncthreads();
            for (int s = tid; s < n; s += kPanelThreads) perm[row_base + rows[s]] = old[s];
        }
    }
    // BF16 staging of L21 (panel rows kmax.. become stage rows 0..), K-major
    if (stage) {
        float *tile = reinterpret_cast<float *>(As);   // 32 rows x kPanelBoMax, reused
        for (int rb = max(r0, kmax); rb < r0 + myR; rb += 32) {
            const int nrow = min(32, r0 + myR - rb);
            __syncthreads();
            for (int e = tid; e < nrow * kmax; e += kPanelThreads) {
                const int r = e % nrow, k = e / nrow;
                tile[(size_t)r * kPanelBoMax + k] = (float)P[(size_t)(rb + r) + (size_t)k * lda];
            }
            __syncthreads();
            for (int e = tid; e < nrow * kpad; e += kPanelThreads) {
                const int r = e / kpad, k = e % kpad;
                const float x = k < kmax ? tile[(size_t)r * kPanelBoMax + k] : 0.f;
                const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                __nv_bfloat16 *dst = stage + (size_t)(rb + r - kmax) * lds;
                dst[k] = hi;
                if (split) dst[kpad + k] = __float2bfloat16_rn(x - __bfloat162float(hi));
            }
        }
    }
    cl.sync();   // no CTA leaves while a peer may still address its shared memory
}

// Rows per CTA and cluster size for an m-row panel (inner width bi, outer bo).
template <typename T>
static bool panel_geometry(int m, int bi, int bo, int max_ctas, size_t smem_cap, int *C_out, int *R_out, size_t *smem_out) {
    auto rows_for = [&](int c) {
        int r = (m + c - 1) / c;
        r = (r + 31) & ~31;
        // the end-of-panel scratch (row map and probe table, or the BF16 tile) reuses As
        const int rmin = (int)((kPanelScratch / (bi * sizeof(T)) + 31) & ~(size_t)31);
        return r > rmin ? r : rmin;
    };
    if (max_ctas < 1 || max_ctas > kPanelMaxCtas) max_ctas = kPanelMaxCtas;
    int C = 1;
    // as many CTAs as allowed while each keeps >= 64 rows: the rank-1 updates are the bulk
    while (C < kPanelMaxCtas && C < max_ctas && (m + 2 * C - 1) / (2 * C) >= 64) C *= 2;
    while (C < kPanelMaxCtas && PanelLayout<T>(rows_for(C), bi, bo, C).total > smem_cap) C *= 2;
    const int R = rows_for(C);
    while (C > 1 && (long long)(C - 1) * R >= m) --C;
    const PanelLayout<T> lay(R, bi, bo, C);
    if (lay.total > smem_cap) return false;
    *C_out = C;
    *R_out = R;
    *smem_out = lay.total;
    return true;
}

// Host launcher: factor the m x bo panel at P with inner width bi; pivots into
// ipiv[0..min(m,bo)) as row_base + local + 1; row map into map_out (may be
// NULL); permutation vector update (may be NULL); optional BF16 staging of
// L21 (stage rows 0.. = panel rows bo..; lds, kpad, split).
template <typename T>
cudaError_t launch_panel_outer(T *P, int lda, int m, int bo, int bi, int *ipiv, int row_base, int *info, int *map_out,
                               int *perm, __nv_bfloat16 *stage, int lds, int kpad, int split, int max_ctas,
                               size_t smem_cap, cudaStream_t s) {
    if (bi <= 0 || bo <= 0 || bo > kPanelBoMax || m <= 0) return cudaErrorInvalidValue;
    if (bi > bo) bi = bo;
    if (bi > kPanelWMax) return cudaErrorInvalidValue;
    int C = 1, R = 0;
    size_t smem = 0;
    if (!panel_geometry<T>(m, bi, bo, max_ctas, smem_cap, &C, &R, &smem)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(panel_factor_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(panel_factor_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kPanelThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    lu_count_launch();
    return cudaLaunchKernelEx(&cfg, panel_factor_cluster<T>, P, lda, m, bo, bi, R, ipiv, row_base, info, map_out, perm,
                              stage, lds, kpad, split);
}

// Largest inner width (power of two, <= cap) for which an m-row panel of outer
// width bo fits on a 16-CTA cluster.
int panel_width_that_fits(int m, size_t elem, size_t smem_cap, int cap, int bo) {
    for (int W = cap; W >= 1; W >>= 1) {
        int C = 0, R = 0;
        size_t sm = 0;
        const int b = bo > 0 ? bo : W;
        const bool ok = elem == 8 ? panel_geometry<double>(m, W, b < W ? W : b, kPanelMaxCtas, smem_cap, &C, &R, &sm)
                                  : panel_geometry<float>(m, W, b < W ? W : b, kPanelMaxCtas, smem_cap, &C, &R, &sm);
        if (ok) return W;
    }
    return 0;
}

template cudaError_t launch_panel_outer<double>(double *, int, int, int, int, int *, int, int *, int *, int *,
                                                __nv_bfloat16 *, int, int, int, int, size_t, cudaStream_t);
template cudaError_t launch_panel_outer<float>(float *, int, int, int, int, int *, int, int *, int *, int *,
                                               __nv_bfloat16 *, int, int, int, int, size_t, cudaStream_t);

}  // namespace lu
