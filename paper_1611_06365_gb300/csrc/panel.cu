// Panel factorization (RL1 / PF3 of the paper) on one thread-block cluster.
//
// One launch factors a whole outer panel of b_o columns (section 3.1,
// Figure 1; the outer/inner split of section 4.2, Figure 6).  The panel's m
// rows are split over the C <= 16 CTAs of a cluster (R rows each), and each
// thread keeps its rows of the current inner panel (b_i <= BI columns) in
// registers: a tile of RPT rows x BI columns (rows tid + 512 u).  Per column j:
//
//   1. every warp finds its (|a|, row) maximum (integer keys: the bits of
//      |a|, compared with warp reductions) and the lane holding it stages
//      that row in shared memory; the thread holding row j stages row j;
//   2. after one CTA barrier every warp knows the CTA's candidate, and all
//      threads PUSH it (key, row index, values) and row j into slots of every
//      CTA of the cluster with asynchronous 16-byte remote stores that count
//      down the destination's transaction barrier (st.async + mbarrier);
//   3. every thread waits on its own CTA's barrier for this column, which
//      completes when all C candidates and row j have landed;
//   4. every warp picks the winner from the slots in its own shared memory
//      (largest magnitude, smallest row on ties); the thread holding row p
//      takes the old row j, the thread holding row j takes the pivot row, and
//      every thread scales its rows of column j by the correctly rounded
//      quotient (FP32: IEEE division; FP64: Markstein's correction from the
//      reciprocal the candidate's warp computed and pushed with the row) and
//      applies the rank-1 update in registers.  The column index is a
//      compile-time constant in that update (one specialised code block per
//      column), so the tile never leaves the register file.
//
// A panel of at most 512 rows (one per thread) whose tile fits one CTA runs
// on a single CTA: its CTA-wide candidate is the pivot, and steps 2 and 3 are
// skipped.
//
// After each inner panel (when b_o > b_i), still inside the same launch:
// its interchanges are applied to the panel's other columns (one row map,
// gather then scatter), U12 := trilu(L11)^{-1} A12 is formed, and the inner
// trailing update A22 -= L21 U12 runs on each thread's rows with L21 taken
// from registers.  At the end the kernel builds the row map of all b_o
// interchanges for the rest of the matrix, updates the permutation vector,
// and, for the tensor-core update, stages L21 in K-major order: BF16,
// BF16 split into hi/lo, or FP8 e4m3 with a power-of-two scale per row.
//
// Early termination (section 4.2): with EtArgs set, the kernel reads a flag at
// the end of each inner panel, after that inner panel's interchanges, U12 and
// inner update have reached the panel's other columns (the right-looking inner
// scheme), and stops there once the step's remainder update has raised it.  The
// columns it leaves are then exactly trailing columns of a step of the width
// it factored; that width is written out and every output (pivots, row map,
// permutation, staging) covers the factored columns only.  CTA 0 reads the flag
// and the other CTAs take its answer from its shared memory, so the whole
// cluster stops at the same boundary.
//
// Slots, staging rows and barriers are double-buffered by column parity: a CTA
// pushes column j+2 only after its barrier for column j+1 completed, i.e.
// after every peer pushed column j+1, which each peer does only after all of
// its threads finished column j (a CTA barrier separates the two).  No
// cluster-wide barrier is needed per column.
#include "common.cuh"
#include "internal.h"
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <climits>
#include <cstddef>

namespace cg = cooperative_groups;

namespace lu {

constexpr int kPanelThreads = 512;
constexpr int kPanelWarps = kPanelThreads / 32;
constexpr int kPanelWMax = 64;       // widest inner panel b_i
constexpr int kPanelBoMax = 256;     // outer panel width b_o
constexpr int kPanelMaxCtas = 16;
constexpr int kPanelTileRegs = 64;   // 32-bit registers per thread for the row tile
constexpr int kPanelMaxRpt = 8;      // rows per thread (R <= 4096)
// end-of-panel scratch: row map (6 b_o ints) + probe table (2 x 4096 ints),
// or the BF16 staging tile (32 rows x b_o floats)
constexpr size_t kPanelScratch = sizeof(int) * (6 * kPanelBoMax + 8192);

// Width BI of the register tile for RPT rows per thread.
template <typename T, int RPT>
struct TileWidth {
    static constexpr int raw = kPanelTileRegs * 4 / (RPT * (int)sizeof(T));
    static constexpr int BI = raw > kPanelWMax ? kPanelWMax : raw;
};

// FP64 scales the panel column by Markstein's correction from a reciprocal that
// the warp holding the candidate computes once (on GB300 an FP64 division costs
// a dozen FP64-pipe operations per row); FP32 divides directly, its division
// being cheap next to the latency a reciprocal would add to the exchange.
template <typename T>
constexpr bool kPanelRcp = sizeof(T) == 8;

template <typename T>
struct __align__(16) CandSlot {
    unsigned long long key;   // magnitude key of the candidate (see mag_key)
    int row;                  // panel row, INT_MAX: no candidate
    int pad;
    T rcp[16 / sizeof(T)];    // [0]: RN(1 / candidate's entry in the current column), FP64 only
    T vals[kPanelWMax];
};

template <typename T>
struct PanelShared {
    CandSlot<T> cand[2][kPanelMaxCtas];      // pushed by every CTA (double-buffered)
    __align__(16) T diag[2][kPanelWMax];     // row j, pushed by its owner
    __align__(16) T wst[2][kPanelWarps][kPanelWMax];   // each warp's candidate row
    T wrcp[2][kPanelWarps];                  // RN(1 / its entry in the current column)
    __align__(16) T jst[2][kPanelWMax];      // row j, staged by its owner
    unsigned long long mbar[2];              // transaction barriers of the column exchange
    unsigned long long red_key[2][kPanelWarps];
    int red_idx[2][kPanelWarps];
    int abort;                               // a wait ran out of time
    int piv[kPanelBoMax];                    // this panel's pivots (panel-local rows)
    int map_rows[2 * kPanelWMax], map_src[2 * kPanelWMax];
    int map_cnt;
    int cnt_s;
    int first_zero;                          // first column with a zero pivot (-1: none)
    int et_stop;                             // CTA 0: stop at this inner boundary
    int kdone;                               // columns factored (fewer after an early termination)
};

// Magnitude key of x: the bits of |x| as an unsigned integer, which orders
// non-negative IEEE values like the values themselves; NaN gets no key
// (the row is not a candidate: NaN never wins a comparison).
__device__ __forceinline__ bool mag_key(float x, unsigned long long &k) {
    const unsigned b = __float_as_uint(x) & 0x7fffffffu;
    k = b;
    return b <= 0x7f800000u;
}
__device__ __forceinline__ bool mag_key(double x, unsigned long long &k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    k = b;
    return b <= 0x7ff0000000000000ULL;
}
__device__ __forceinline__ bool key_better(unsigned long long ka, int ia, unsigned long long kb, int ib) {
    return ka > kb || (ka == kb && ia < ib);
}

// Warp-wide (key, row) maximum, smallest row on ties; every lane gets the
// result.  No candidate: key 0, row INT_MAX (loses to any real row).
__device__ __forceinline__ void warp_argmax_key(unsigned long long &key, int &idx) {
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    const unsigned mine = (hi == mh && lo == ml) ? (unsigned)idx : 0xffffffffu;
    idx = (int)__reduce_min_sync(0xffffffffu, mine);
    key = ((unsigned long long)mh << 32) | ml;
}

// The same for keys that fit in 32 bits (FP32 magnitudes): two reductions.
__device__ __forceinline__ void warp_argmax_key32(unsigned long long &key, int &idx) {
    const unsigned k32 = (unsigned)key;
    const unsigned mk = __reduce_max_sync(0xffffffffu, k32);
    idx = (int)__reduce_min_sync(0xffffffffu, k32 == mk ? (unsigned)idx : 0xffffffffu);
    key = mk;
}
template <typename T>
__device__ __forceinline__ void warp_argmax_t(unsigned long long &key, int &idx) {
    if constexpr (sizeof(T) == 4) warp_argmax_key32(key, idx);
    else warp_argmax_key(key, idx);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned peer_u32(unsigned a, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// 16-byte asynchronous store into a peer's shared memory; its completion
// counts 16 bytes down on the peer's transaction barrier.
__device__ __forceinline__ void st_async16(unsigned peer_addr, int4 v, unsigned peer_mbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(peer_addr),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"(peer_mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(unsigned mb, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned mb, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of the barrier at mb.  After `bound_ns` of
// globaltimer time it records LU_ERR_TIMEOUT, marks the CTA aborted (later
// waits return at once) and returns: the kernel then runs to its end with
// meaningless values but keeps every CTA's control flow, so no barrier hangs.
__device__ __forceinline__ void mbar_wait_bounded(unsigned mb, unsigned parity, volatile int *abort, int *status,
                                                  long long bound_ns) {
    if (*abort) return;
    unsigned spins = 0;
    unsigned long long t0 = 0;
    while (!mbar_try_wait(mb, parity)) {
        if ((++spins & 63u) == 0u) {
            const unsigned long long t = lu_globaltimer();
            if (t0 == 0) {
                t0 = t;
            } else if ((long long)(t - t0) > bound_ns) {
                *abort = 1;
                if (status) atomicExch(status, (int)LU_ERR_TIMEOUT);
                return;
            }
            if (*abort) return;
        }
    }
}

// Dynamic shared memory: PanelShared | scratch | U12s[bo-1][bi+1] | gv[ceil(bo/C)][2 bi] | L11s[bi][bi]
template <typename T>
struct PanelLayout {
    size_t scratch_off, u12_off, gv_off, l11_off, total;
    __host__ __device__ PanelLayout(int bi, int bo, int C) {
        scratch_off = (sizeof(PanelShared<T>) + 15) & ~(size_t)15;
        u12_off = scratch_off + ((kPanelScratch + 15) & ~(size_t)15);
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

// 16-byte vector type for T
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

// Tile row uu (runtime, < RPT) into dst[0..BI) (16-byte aligned shared memory).
template <typename T, int RPT, int BI>
__device__ __forceinline__ void stage_tile_row(const T (&a)[RPT][BI], int uu, T *dst) {
    using V = typename Vec16<T>::type;
    constexpr int VEC = 16 / sizeof(T);
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        if (u != uu) continue;
#pragma unroll
        for (int q = 0; q < BI / VEC; ++q) {
            T w[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) w[k] = a[u][q * VEC + k];
            reinterpret_cast<V *>(dst)[q] = *reinterpret_cast<const V *>(w);
        }
    }
}

// Column step LJ (a compile-time constant) of the rank-1 update on this
// thread's rows below row j: a(i, LJ) /= pv, a(i, c) -= a(i, LJ) u(c) for
// c > LJ, and the candidate of column LJ + 1 (when LJ + 1 < wi).
template <typename T, int RPT, int BI, int LJ>
__device__ __forceinline__ void rank1_step(T (&a)[RPT][BI], const T *__restrict__ urow, T pv, T rcp, bool zero, int tid,
                                           int r0, int myR, int j, int wi, unsigned long long &best, int &bidx) {
    using V = typename Vec16<T>::type;
    constexpr int VEC = 16 / sizeof(T);
    constexpr int Q0 = (LJ + 1) / VEC;   // first vector of urow holding a column > LJ
    bool act[RPT];
    T l[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int lr = tid + u * kPanelThreads;
        act[u] = (lr < myR) && (r0 + lr > j) && !zero;
        l[u] = T(0);
        if (act[u]) {
            const T x = a[u][LJ];
            if constexpr (kPanelRcp<T>) {
                // the correctly rounded x / pv from the pivot's reciprocal (Markstein's
                // correction), IEEE division where an operand is outside its safe range
                l[u] = lu_div_safe(x, lu_div_range<T>::in(pv)) ? lu_div_fast(x, pv, rcp) : x / pv;
            } else {
                l[u] = x / pv;
            }
            a[u][LJ] = l[u];
        }
    }
#pragma unroll
    for (int q = Q0; q < BI / VEC; ++q) {
        V vv = reinterpret_cast<const V *>(urow)[q];
        const T *w = reinterpret_cast<const T *>(&vv);
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            const int c = q * VEC + k;
            if (c > LJ) {
#pragma unroll
                for (int u = 0; u < RPT; ++u)
                    if (act[u]) a[u][c] = fma(-l[u], w[k], a[u][c]);
            }
        }
    }
    best = 0;
    bidx = INT_MAX;
    if constexpr (LJ + 1 < BI) {
        if (LJ + 1 < wi) {
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                const int lr = tid + u * kPanelThreads, i = r0 + lr;
                unsigned long long k;
                if (lr < myR && i > j && mag_key(a[u][LJ + 1], k) && key_better(k, i, best, bidx)) { best = k; bidx = i; }
            }
        }
    }
}

#define LU_PANEL_CASE(L)                                                                                   \
    case (L):                                                                                              \
        if constexpr ((L) < BI)                                                                            \
            rank1_step<T, RPT, BI, ((L) < BI ? (L) : 0)>(a, urow, pv, rcp, zero, tid, r0, myR, j, wi, best, bidx); \
        break;
#define LU_PANEL_CASE4(L) LU_PANEL_CASE(L) LU_PANEL_CASE((L) + 1) LU_PANEL_CASE((L) + 2) LU_PANEL_CASE((L) + 3)
#define LU_PANEL_CASE16(L) LU_PANEL_CASE4(L) LU_PANEL_CASE4((L) + 4) LU_PANEL_CASE4((L) + 8) LU_PANEL_CASE4((L) + 12)

template <typename T, int RPT, bool ET>
__global__ void __launch_bounds__(kPanelThreads, 1)
panel_factor_cluster(T *__restrict__ P, int lda, int m, int bo, int bi, int R, int *__restrict__ ipiv, int row_base,
                     int *__restrict__ info, int *__restrict__ map_out, int *__restrict__ perm,
                     StageDesc sd, int *__restrict__ status, long long bound_ns, CtaTrace tr, int *__restrict__ yreq,
                     EtArgs et) {
    const unsigned long long t_start = tr.ring ? lu_globaltimer() : 0ull;
    constexpr int BI = TileWidth<T, RPT>::BI;
    using V = typename Vec16<T>::type;
    constexpr int VEC = 16 / sizeof(T);
    static_assert(BI % VEC == 0, "tile width must be a whole number of 16-byte vectors");
    static_assert(offsetof(CandSlot<T>, rcp) == 16 && offsetof(CandSlot<T>, vals) == 32,
                  "the exchange writes a candidate slot as 16-byte vectors: header, reciprocal, row");
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // the cluster is in: a persistent update no longer needs to give SMs back
    if (yreq && rank == 0 && tid == 0) atomicExch(yreq, 0);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PanelLayout<T> lay(bi, bo, C);
    PanelShared<T> &S = *reinterpret_cast<PanelShared<T> *>(smem_raw);
    unsigned char *scratch = smem_raw + lay.scratch_off;
    T *U12s = reinterpret_cast<T *>(smem_raw + lay.u12_off);
    T *gv = reinterpret_cast<T *>(smem_raw + lay.gv_off);
    T *L11s = reinterpret_cast<T *>(smem_raw + lay.l11_off);   // [wi][wi] column-major, inner transitions

    const int r0 = rank * R;
    const int myR = max(0, min(R, m - r0));
    const int kmax = min(m, bo);
    if (tid == 0) {
        S.first_zero = -1;
        S.kdone = kmax;
        S.abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cl.sync();   // every CTA has started and initialised its barriers before any remote store

    T a[RPT][BI];   // rows r0 + tid + 512 u of the inner panel's columns

    for (int jb = 0; jb < kmax; jb += bi) {
        const int wi = min(bi, kmax - jb);
        // (a) own rows at or below the inner panel into registers (coalesced down each column)
        unsigned long long best = 0;
        int bidx = INT_MAX;
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int lr = tid + u * kPanelThreads, i = r0 + lr;
            const bool ld = (lr < myR) && (i >= jb);
#pragma unroll
            for (int c = 0; c < BI; ++c) a[u][c] = (ld && c < wi) ? P[(size_t)i + (size_t)(jb + c) * lda] : T(0);
            unsigned long long k;
            if (ld && mag_key(a[u][0], k) && key_better(k, i, best, bidx)) { best = k; bidx = i; }
        }
        // (b) column steps: one CTA barrier and one cluster exchange per column
        const int nvec = (wi + VEC - 1) / VEC;
        // bytes landing in each CTA per column: C headers (and reciprocals) and
        // candidate rows, one row j
        constexpr int qoff = kPanelRcp<T> ? 2 : 1;   // 16-byte vectors before a candidate row
        const unsigned xbytes = 16u * (unsigned)(C * (qoff + nvec) + nvec);
        for (int lj = 0; lj < wi; ++lj) {
            const int j = jb + lj;
            const int par = j & 1;
            const unsigned mb = smem_u32(&S.mbar[par]);
            if (C > 1 && tid == 0) mbar_arrive_expect(mb, xbytes);
            warp_argmax_t<T>(best, bidx);
            // the lane holding the warp's candidate stages it; the owner of row j stages row j
            // (FP64: with the reciprocal of its entry in column j, one division per
            // warp instead of one per row)
            if (bidx != INT_MAX && lane == ((bidx - r0) & 31)) {
                stage_tile_row<T, RPT, BI>(a, (bidx - r0) / kPanelThreads, S.wst[par][warp]);
                if constexpr (kPanelRcp<T>) S.wrcp[par][warp] = T(1) / S.wst[par][warp][lj];
            }
            const bool own_j = (j >= r0 && j < r0 + myR);
            if (own_j && tid == (j - r0) % kPanelThreads)
                stage_tile_row<T, RPT, BI>(a, (j - r0) / kPanelThreads, S.jst[par]);
            if (lane == 0) { S.red_key[par][warp] = best; S.red_idx[par][warp] = bidx; }
            __syncthreads();
            // every warp reduces the warp candidates itself (no second barrier)
            unsigned long long ckey = lane < kPanelWarps ? S.red_key[par][lane] : 0ULL;
            int crow = lane < kPanelWarps ? S.red_idx[par][lane] : INT_MAX;
            warp_argmax_t<T>(ckey, crow);
            const T *urow;
            const T *drow = S.jst[par];    // old row j, the new content of row p
            int p;
            bool valid;
            T rcp;
            if (C == 1) {
                // one CTA holds every row: its candidate is the pivot, no exchange
                valid = (crow != INT_MAX);
                p = valid ? crow : j;
                const int w = ((crow - r0) >> 5) & (kPanelWarps - 1);
                urow = valid ? S.wst[par][w] : S.jst[par];
                if constexpr (kPanelRcp<T>) rcp = valid ? S.wrcp[par][w] : T(1) / urow[lj];
                else rcp = T(0);
            } else {
                // push header, reciprocal, candidate row and row j into every CTA, 16 bytes per store
                const int ndiag = own_j ? nvec : 0;
                const int per = qoff + nvec + ndiag;
                const int cw = crow != INT_MAX ? ((crow - r0) >> 5) & (kPanelWarps - 1) : 0;
                const int4 *crow_src = reinterpret_cast<const int4 *>(S.wst[par][cw]);
                const unsigned slot = smem_u32(&S.cand[par][rank]);
                const unsigned dslot = smem_u32(S.diag[par]);
                for (int e = tid; e < C * per; e += kPanelThreads) {
                    const int d = e / per, q = e % per;
                    int4 v;
                    unsigned addr;
                    if (q == 0) {
                        v = make_int4((int)(unsigned)ckey, (int)(unsigned)(ckey >> 32), crow, 0);
                        addr = slot;
                    } else if (kPanelRcp<T> && q == 1) {
                        T rv[16 / sizeof(T)] = {};
                        rv[0] = crow != INT_MAX ? S.wrcp[par][cw] : T(0);
                        v = *reinterpret_cast<const int4 *>(rv);
                        addr = slot + 16u;
                    } else if (q < qoff + nvec) {
                        v = crow_src[q - qoff];
                        addr = slot + 32u + 16u * (unsigned)(q - qoff);
                    } else {
                        v = reinterpret_cast<const int4 *>(S.jst[par])[q - qoff - nvec];
                        addr = dslot + 16u * (unsigned)(q - qoff - nvec);
                    }
                    st_async16(peer_u32(addr, d), v, peer_u32(mb, d));
                }
                mbar_wait_bounded(mb, (unsigned)(j >> 1) & 1u, &S.abort, status, bound_ns);
                // winner from the local copies, reduced by every warp (no barrier)
                const int4 hdr = lane < C ? *reinterpret_cast<const int4 *>(&S.cand[par][lane]) : make_int4(0, 0, INT_MAX, 0);
                unsigned long long wk = ((unsigned long long)(unsigned)hdr.y << 32) | (unsigned)hdr.x;
                int ix = hdr.z;
                const int mine = ix;
                warp_argmax_t<T>(wk, ix);
                valid = (ix != INT_MAX);
                const int src = valid ? __ffs(__ballot_sync(0xffffffffu, mine == ix)) - 1 : 0;
                p = valid ? ix : j;   // every candidate NaN: keep row j, as a sequential scan would
                urow = valid ? S.cand[par][src].vals : S.diag[par];
                drow = S.diag[par];
                if constexpr (kPanelRcp<T>) rcp = valid ? S.cand[par][src].rcp[0] : T(1) / urow[lj];
                else rcp = T(0);
            }
            const T pv = urow[lj];
            const bool zero = (pv == T(0));
            if (tid == 0) {
                S.piv[j] = zero ? j : p;
                if (zero && S.first_zero < 0) S.first_zero = j;
            }
            // the interchange: row j takes the pivot row, row p the old row j
            // (whole rows of the inner panel, factored columns included)
            if (!zero && p != j) {
#pragma unroll
                for (int u = 0; u < RPT; ++u) {
                    const int lr = tid + u * kPanelThreads;
                    if (lr >= myR) continue;
                    const int i = r0 + lr;
                    if (i == j || i == p) {
                        const V *s = reinterpret_cast<const V *>(i == j ? urow : drow);
#pragma unroll
                        for (int q = 0; q < BI / VEC; ++q) {
                            V vv = s[q];
                            const T *w = reinterpret_cast<const T *>(&vv);
#pragma unroll
                            for (int k = 0; k < VEC; ++k) a[u][q * VEC + k] = w[k];
                        }
                    }
                }
            }
            // scaling and rank-1 update with the column index as a constant
            switch (lj) {
                LU_PANEL_CASE16(0)
                LU_PANEL_CASE16(16)
                LU_PANEL_CASE16(32)
                LU_PANEL_CASE16(48)
                default: break;
            }
        }
        // (c) the factored inner panel back to global memory (rows at or below jb)
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int lr = tid + u * kPanelThreads, i = r0 + lr;
            if (lr >= myR || i < jb) continue;
#pragma unroll
            for (int c = 0; c < BI; ++c)
                if (c < wi) P[(size_t)i + (size_t)(jb + c) * lda] = a[u][c];
        }
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
            // (f) inner update of this thread's rows below the inner panel,
            // A22 -= L21 U12, with L21 from registers (4 columns at a time)
#pragma unroll
            for (int u = 0; u < RPT; ++u) {
                const int lr = tid + u * kPanelThreads, i = r0 + lr;
                if (lr >= myR || i < c_right) continue;
                T *row = P + (size_t)i + (size_t)c_right * lda;
                for (int c = 0; c < nr; c += 4) {
                    T acc[4] = {T(0), T(0), T(0), T(0)};
                    T old[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) old[v] = c + v < nr ? row[(size_t)(c + v) * lda] : T(0);
#pragma unroll
                    for (int kk = 0; kk < BI; ++kk) {
                        if (kk < wi) {
#pragma unroll
                            for (int v = 0; v < 4; ++v)
                                if (c + v < nr) acc[v] = fma(a[u][kk], U12s[(size_t)(c + v) * (wi + 1) + kk], acc[v]);
                        }
                    }
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        if (c + v < nr) row[(size_t)(c + v) * lda] = old[v] - acc[v];
                }
            }
        }
        cl.sync();
        // early termination: stop here once the step's remainder update is done
        if (ET && c_right < kmax) {
            if (rank == 0 && tid == 0) S.et_stop = et.force ? 1 : (lu_ld_acquire(et.flag) == et.epoch ? 1 : 0);
            cl.sync();
            if (*cl.map_shared_rank(&S.et_stop, 0)) {
                if (tid == 0) S.kdone = c_right;
                break;
            }
        }
    }
    cl.sync();   // all of the panel is final in global memory
    const int kdone = ET ? S.kdone : kmax;
    // pivots and the first zero pivot, written once per panel
    if (rank == 0) {
        for (int j = tid; j < kdone; j += kPanelThreads) ipiv[j] = row_base + S.piv[j] + 1;
        if (tid == 0 && S.first_zero >= 0) atomicCAS(info, 0, row_base + S.first_zero + 1);
        if (tid == 0 && et.w_out) *et.w_out = kdone;
    }

    // row map of all the panel's interchanges, for the rest of the matrix:
    // [0] count, [1 .. 1+2b) rows, [1+2b .. 1+4b) src (matrix rows), b = kdone
    // (bo unless the panel stopped early)
    if (rank == 0 && map_out) {
        int *rows = reinterpret_cast<int *>(scratch);
        int *src = rows + 2 * kPanelBoMax;
        int *old = src + 2 * kPanelBoMax;
        int *keys = old + 2 * kPanelBoMax;
        int *slot = keys + 4096;
        for (int i = tid; i < 4096; i += kPanelThreads) keys[i] = -1;
        __syncthreads();
        if (tid == 0) {
            int n = kdone;
            for (int t = 0; t < kdone; ++t) { rows[t] = t; src[t] = t; }
            for (int j = 0; j < kdone; ++j) {
                const int q = S.piv[j];
                if (q == j) continue;
                int iq;
                if (q < kdone) {
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
            map_out[1 + 2 * kdone + s] = row_base + src[s];
        }
        if (perm) {
            for (int s = tid; s < n; s += kPanelThreads) old[s] = perm[row_base + src[s]];
            __syncthreads();
            for (int s = tid; s < n; s += kPanelThreads) perm[row_base + rows[s]] = old[s];
        }
    }
    // staging of L21 for the tensor-core update (panel rows kdone.. become stage
    // rows 0..), K-major, in 32-row chunks through shared memory
    if constexpr (sizeof(T) == 8) {
        if (sd.ptr && sd.fmt == 3) {
            // FP64 digit slices (emulated FP64 update; kdone <= kpad = 64): one power-of-two
            // scale per row from the row's largest magnitude, 16 threads per row
            T *tile = reinterpret_cast<T *>(scratch);                 // 32 rows x 64
            int *rexp = reinterpret_cast<int *>(tile + 32 * 64);
            __nv_bfloat16 *st16 = static_cast<__nv_bfloat16 *>(sd.ptr);
            for (int rb = max(r0, kdone); rb < r0 + myR; rb += 32) {
                const int nrow = min(32, r0 + myR - rb);
                __syncthreads();
                for (int e = tid; e < nrow * kdone; e += kPanelThreads) {
                    const int r = e % nrow, k = e / nrow;
                    tile[(size_t)r * 64 + k] = P[(size_t)(rb + r) + (size_t)k * lda];
                }
                __syncthreads();
                {
                    const int r = tid >> 4, sub = tid & 15;
                    unsigned long long amax = 0;
                    if (r < nrow)
                        for (int k = sub; k < kdone; k += 16) amax = max(amax, lu_f64_abs_bits(tile[(size_t)r * 64 + k]));
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                    if (sub == 0 && r < nrow) {
                        const int ex = lu_f64_scale_exp_bits(amax);
                        rexp[r] = ex;
                        sd.dscale[rb + r - kdone] = ldexp(1.0, ex);
                    }
                }
                __syncthreads();
                for (int e = tid; e < nrow * sd.kpad; e += kPanelThreads) {
                    const int r = e / sd.kpad, k = e % sd.kpad;
                    lu_f64_slices(k < kdone ? tile[(size_t)r * 64 + k] : 0.0, rexp[r],
                                  st16 + (size_t)(rb + r - kdone) * sd.lds + k, (size_t)sd.kpad);
                }
            }
        }
    }
    if (sd.ptr && sd.fmt != 3) {
        float *tile = reinterpret_cast<float *>(scratch);   // 32 rows x kPanelBoMax, reused
        float *rowmul = tile + 32 * kPanelBoMax;              // FP8: the rows' scale factors
        const int kpad = sd.kpad;
        for (int rb = max(r0, kdone); rb < r0 + myR; rb += 32) {
            const int nrow = min(32, r0 + myR - rb);
            __syncthreads();
            for (int e = tid; e < nrow * kdone; e += kPanelThreads) {
                const int r = e % nrow, k = e / nrow;
                tile[(size_t)r * kPanelBoMax + k] = (float)P[(size_t)(rb + r) + (size_t)k * lda];
            }
            __syncthreads();
            if (sd.fmt == 2) {
                // one power-of-two scale per row: 16 threads per row reduce |x|
                const int r = tid >> 4, sub = tid & 15;
                float amax = 0.f;
                if (r < nrow)
                    for (int k = sub; k < kdone; k += 16) amax = fmaxf(amax, fabsf(tile[(size_t)r * kPanelBoMax + k]));
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                float inv;
                const float mul = lu_fp8_scale(amax, &inv);
                if (sub == 0 && r < nrow) {
                    rowmul[r] = mul;
                    sd.scale[rb + r - kdone] = inv;
                }
                __syncthreads();
                unsigned char *st8 = static_cast<unsigned char *>(sd.ptr);
                for (int e = tid; e < nrow * kpad; e += kPanelThreads) {
                    const int rr = e / kpad, k = e % kpad;
                    st8[(size_t)(rb + rr - kdone) * sd.lds + k] =
                        k < kdone ? lu_to_e4m3(tile[(size_t)rr * kPanelBoMax + k] * rowmul[rr]) : (unsigned char)0;
                }
            } else {
                __nv_bfloat16 *st16 = static_cast<__nv_bfloat16 *>(sd.ptr);
                for (int e = tid; e < nrow * kpad; e += kPanelThreads) {
                    const int r = e / kpad, k = e % kpad;
                    const float x = k < kdone ? tile[(size_t)r * kPanelBoMax + k] : 0.f;
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    __nv_bfloat16 *dst = st16 + (size_t)(rb + r - kdone) * sd.lds;
                    dst[k] = hi;
                    if (sd.fmt == 1) dst[kpad + k] = __float2bfloat16_rn(x - __bfloat162float(hi));
                }
            }
        }
    }
    cl.sync();   // no CTA leaves while a peer may still address its shared memory
    if (tid == 0) lu_trace_cta(tr, t_start, 0);
}

// Rows per thread for a CTA of R rows (a power of two).
static int rows_per_thread(int R) {
    int r = 1;
    while (r * kPanelThreads < R) r *= 2;
    return r;
}

template <typename T>
static int tile_width(int rpt) {
    switch (rpt) {
        case 1: return TileWidth<T, 1>::BI;
        case 2: return TileWidth<T, 2>::BI;
        case 4: return TileWidth<T, 4>::BI;
        case 8: return TileWidth<T, 8>::BI;
        default: return 0;
    }
}

// Cluster size C and rows per CTA R for an m-row panel of inner width bi:
// as many CTAs as allowed while each keeps >= 64 rows, more when the
// register tile cannot hold R rows at width bi.
template <typename T>
static bool panel_geometry(int m, int bi, int bo, int max_ctas, size_t smem_cap, int *C_out, int *R_out, size_t *smem_out) {
    auto rows_for = [&](int c) {
        const int r = (m + c - 1) / c;
        return (r + 31) & ~31;
    };
    auto fits = [&](int c) {
        const int rpt = rows_per_thread(rows_for(c));
        return rpt <= kPanelMaxRpt && tile_width<T>(rpt) >= bi;
    };
    if (max_ctas < 1 || max_ctas > kPanelMaxCtas) max_ctas = kPanelMaxCtas;
    int C = 1;
    // up to one row per thread, one CTA holds the panel (no cluster exchange per
    // column) when its tile and its share of the other columns fit
    if (m > kPanelThreads || tile_width<T>(1) < bi || PanelLayout<T>(bi, bo, 1).total > smem_cap)
        while (C < kPanelMaxCtas && C < max_ctas && (m + 2 * C - 1) / (2 * C) >= 64) C *= 2;
    while (C < kPanelMaxCtas && !fits(C)) C *= 2;
    if (!fits(C)) return false;
    const int R = rows_for(C);
    while (C > 1 && (long long)(C - 1) * R >= m) --C;
    const PanelLayout<T> lay(bi, bo, C);
    if (lay.total > smem_cap) return false;
    *C_out = C;
    *R_out = R;
    *smem_out = lay.total;
    return true;
}

template <typename T, int RPT>
static cudaError_t launch_rpt(cudaLaunchConfig_t &cfg, T *P, int lda, int m, int bo, int bi, int R, int *ipiv,
                              int row_base, int *info, int *map_out, int *perm, StageDesc sd, int *status, long long bound_ns,
                              const CtaTrace &tr, int *yreq, const EtArgs &et) {
    // the early-termination check is compiled only into the variant that uses it
    auto kern = (et.flag || et.force) ? panel_factor_cluster<T, RPT, true> : panel_factor_cluster<T, RPT, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.dynamicSmemBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    lu_count_launch();
    return cudaLaunchKernelEx(&cfg, kern, P, lda, m, bo, bi, R, ipiv, row_base, info, map_out, perm, sd, status, bound_ns,
                              tr, yreq, et);
}

// Host launcher: factor the m x bo panel at P with inner width bi; pivots into
// ipiv[0..min(m,bo)) as row_base + local + 1; row map into map_out (may be
// NULL); permutation vector update (may be NULL); optional BF16 staging of
// L21 (stage rows 0.. = panel rows bo.., as described by sd).  A column
// exchange that waits longer than bound_ns records LU_ERR_TIMEOUT in *status.
// yreq (may be NULL): the worker-sharing request (SmShare), cleared once the
// cluster runs.  et: early termination at an inner boundary (EtArgs); the
// factored width is then written to *et.w_out and the row map is laid out
// for that width.
template <typename T>
cudaError_t launch_panel_outer(T *P, int lda, int m, int bo, int bi, int *ipiv, int row_base, int *info, int *map_out,
                               int *perm, StageDesc sd, int max_ctas, size_t smem_cap, int *status, long long bound_ns,
                               cudaStream_t s, CtaTrace tr, int *yreq, EtArgs et) {
    if (bi <= 0 || bo <= 0 || bo > kPanelBoMax || m <= 0) return cudaErrorInvalidValue;
    if (bi > bo) bi = bo;
    if (bi > kPanelWMax) return cudaErrorInvalidValue;
    int C = 1, R = 0;
    size_t smem = 0;
    if (!panel_geometry<T>(m, bi, bo, max_ctas, smem_cap, &C, &R, &smem)) return cudaErrorInvalidValue;
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
    switch (rows_per_thread(R)) {
        case 1: return launch_rpt<T, 1>(cfg, P, lda, m, bo, bi, R, ipiv, row_base, info, map_out, perm, sd, status, bound_ns, tr, yreq, et);
        case 2: return launch_rpt<T, 2>(cfg, P, lda, m, bo, bi, R, ipiv, row_base, info, map_out, perm, sd, status, bound_ns, tr, yreq, et);
        case 4: return launch_rpt<T, 4>(cfg, P, lda, m, bo, bi, R, ipiv, row_base, info, map_out, perm, sd, status, bound_ns, tr, yreq, et);
        case 8: return launch_rpt<T, 8>(cfg, P, lda, m, bo, bi, R, ipiv, row_base, info, map_out, perm, sd, status, bound_ns, tr, yreq, et);
        default: return cudaErrorInvalidValue;
    }
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

// Whether launch_panel_outer accepts an m-row panel of outer width bo and inner width bi.
bool panel_fits(int m, size_t elem, int bo, int bi, int max_ctas, size_t smem_cap) {
    int C = 0, R = 0;
    size_t sm = 0;
    return elem == 8 ? panel_geometry<double>(m, bi, bo, max_ctas, smem_cap, &C, &R, &sm)
                     : panel_geometry<float>(m, bi, bo, max_ctas, smem_cap, &C, &R, &sm);
}

// CTAs of the cluster launch_panel_outer makes for these arguments (0: it
// would refuse them).
int panel_cluster_ctas(int m, size_t elem, int bo, int bi, int max_ctas, size_t smem_cap) {
    if (bi > bo) bi = bo;
    int C = 0, R = 0;
    size_t sm = 0;
    const bool ok = elem == 8 ? panel_geometry<double>(m, bi, bo, max_ctas, smem_cap, &C, &R, &sm)
                              : panel_geometry<float>(m, bi, bo, max_ctas, smem_cap, &C, &R, &sm);
    return ok ? C : 0;
}

// ---- worker sharing (SmShare) ----------------------------------------------

// One cluster of C CTAs marks the SMs it was placed on: a set of SMs that can
// hold a panel cluster of that size (clusters stay within one GPC).
__global__ void cluster_sm_probe(unsigned *mask) {
    if (threadIdx.x == 0) {
        const unsigned s = lu_smid();
        if (s < kShareMaskBits) atomicOr(&mask[s >> 5], 1u << (s & 31u));
        else atomicOr(&mask[kShareMaskBits / 32], 1u);   // an id the mask cannot hold: sharing stays off
    }
}

cudaError_t launch_cluster_sm_probe(int C, unsigned *mask, cudaStream_t s) {
    if (C < 1 || C > kPanelMaxCtas) return cudaErrorInvalidValue;
    if (C > 8) {
        cudaError_t e = cudaFuncSetAttribute(cluster_sm_probe, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(32, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    lu_count_launch();
    return cudaLaunchKernelEx(&cfg, cluster_sm_probe, mask);
}

__global__ void share_raise(int *req) { *req = 1; }

// The panel branch asks for its SMs back (runs just before the panel).
cudaError_t launch_share_raise(int *req, cudaStream_t s) {
    share_raise<<<1, 1, 0, s>>>(req);
    lu_count_launch();
    return cudaGetLastError();
}

// ---- early termination -------------------------------------------------------

// The remainder update of step k is done: raise the flag panel k+1 reads at its
// inner boundaries (section 4.2: written only by the update side, read only by
// the panel side).
__global__ void et_signal(int *flag, int epoch) { lu_st_release(flag, epoch); }

cudaError_t launch_et_signal(int *flag, int epoch, cudaStream_t s) {
    et_signal<<<1, 1, 0, s>>>(flag, epoch);
    lu_count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_panel_outer<double>(double *, int, int, int, int, int *, int, int *, int *, int *, StageDesc,
                                                int, size_t, int *, long long, cudaStream_t, CtaTrace, int *, EtArgs);
template cudaError_t launch_panel_outer<float>(float *, int, int, int, int, int *, int, int *, int *, int *, StageDesc, int,
                                               size_t, int *, long long, cudaStream_t, CtaTrace, int *, EtArgs);

}  // namespace lu
