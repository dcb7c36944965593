// C ABI of liblu (declared in include/lu.h) and the host-side scheduler of the
// blocked right-looking LU with look-ahead.
//
// Schedule (section 3.2, Figure 3; section 4.1 for worker sharing).  Two
// streams per device: P (highest priority) carries the panel branch T_PF and
// U (lowest priority) the remainder branch T_RU.  For outer iteration k
// (panel k already factored on P, its interchanges in row map k):
//
//   U:  wait panel(k) | interchanges on the columns left of panel k |
//       RU1: interchanges + TRSM on the columns right of strip k+1 |
//       RU2: update of those columns
//   P:  wait RU2(k-1) | PF1: interchanges + TRSM on strip k+1 |
//       PF2: update of strip k+1 | PF3: factor panel k+1 (cluster kernel)
//
// No kernel waits on another kernel: the branches are ordered with CUDA
// events only.  Worker sharing comes from the GPU's CTA scheduler: RU2 is a
// grid with many more tiles than SMs, so when the panel cluster exits its SMs
// are handed the RU2 tiles still queued -- the GPU counterpart of the paper's
// malleable BLAS, where PF threads join RU2 at the next Loop-4 boundary.
//
// An outer panel wider than what one cluster holds in shared memory is
// factored by the inner/outer scheme of section 4.2 (Figure 6): inner panels
// of width b_i on the cluster, each followed by its interchanges, TRSM and
// update restricted to the outer panel.
//
// Early termination (section 4.2, lu_opts.early_term): after RU2(k) a
// one-thread kernel raises a flag on U; panel k+1 reads it at the end of
// each inner panel and stops there, leaving the rest of its strip in the
// state of trailing columns after a step of the width it reached.  The host
// reads that width back before it enqueues step k+1, whose strip then takes
// step k+1 only beyond panel k+1's nominal columns.
//
// Plans: b_o, b_i, the panel team and the RU2 grid come from lu_opts, else
// from the autotuner's table (tune.cu), else from the built-in choice
// (make_plan); every panel of a plan is checked to fit a cluster before
// anything is enqueued.
#include "common.cuh"
#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

using namespace lu;

// ---------------------------------------------------------------------------
// per-device state
// ---------------------------------------------------------------------------
namespace {

constexpr int kMaxDev = 64;
constexpr size_t kPanelSmemCap = 200 * 1024;
constexpr int kMaxDepth = 4;              // deepest look-ahead (lu_opts.lookahead)
constexpr int kRing = kMaxDepth + 1;      // panels whose row maps / staging may be in use at once

constexpr int kMaskWords = kShareMaskBits / 32 + 1;   // SM bits, then an overflow word

struct DevState {
    bool init = false;
    cudaStream_t P = nullptr, U = nullptr;
    cudaStream_t J = nullptr;   // joining grids of the remainder update (worker sharing)
    cudaEvent_t evP[kRing] = {}, evU[kRing] = {};
    cudaEvent_t evIn = nullptr, evOutP = nullptr, evOutU = nullptr, evPF2 = nullptr;
    cudaEvent_t evPanelEnd = nullptr, evGo = nullptr, evJ = nullptr;
    int *status = nullptr;   // device status word
    int *share_req = nullptr;        // SmShare request word
    unsigned *share_mask = nullptr;  // [17][kMaskWords]: SMs of one cluster placement of C CTAs
    signed char share_state[17] = {};   // per C: 0 not probed, 1 probed, -1 probe refused
    int sms = 0;
    int *et = nullptr;               // early termination: [0] flag, [1] width the panel reached
    std::vector<int> widths;         // panel widths of the last factorization
    bool widths_valid = false;
};

DevState g_dev[kMaxDev];
std::mutex g_mu;
std::recursive_mutex g_enqueue_mu;   // the per-device streams/events serve one enqueue at a time
char g_last_err[512];

cudaError_t dev_state(DevState **out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &st = g_dev[d];
    if (!st.init) {
        int lo = 0, hi = 0;
        if ((e = cudaDeviceGetStreamPriorityRange(&lo, &hi)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithPriority(&st.P, cudaStreamNonBlocking, hi)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithPriority(&st.U, cudaStreamNonBlocking, lo)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithPriority(&st.J, cudaStreamNonBlocking, lo)) != cudaSuccess) return e;
        for (int i = 0; i < kRing; ++i) {
            if ((e = cudaEventCreateWithFlags(&st.evP[i], cudaEventDisableTiming)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&st.evU[i], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        if ((e = cudaEventCreateWithFlags(&st.evIn, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&st.evOutP, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&st.evOutU, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&st.evPF2, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&st.evPanelEnd, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&st.evGo, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&st.evJ, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&st.status, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemset(st.status, 0, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&st.share_req, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemset(st.share_req, 0, sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&st.share_mask, 17 * kMaskWords * sizeof(unsigned))) != cudaSuccess) return e;
        if ((e = cudaMemset(st.share_mask, 0, 17 * kMaskWords * sizeof(unsigned))) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&st.sms, cudaDevAttrMultiProcessorCount, d)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&st.et, 2 * sizeof(int))) != cudaSuccess) return e;
        if ((e = cudaMemset(st.et, 0, 2 * sizeof(int))) != cudaSuccess) return e;
        st.init = true;
    }
    *out = &st;
    return cudaSuccess;
}

// stream-ordered workspace that is released on the caller's stream
struct Workspace {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Workspace(cudaStream_t st) : s(st) {}
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        void *v = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMallocAsync(&v, count * sizeof(T), s);
        if (e != cudaSuccess) return e;
        ptrs.push_back(v);
        *p = static_cast<T *>(v);
        return cudaSuccess;
    }
    ~Workspace() {
        for (void *v : ptrs) cudaFreeAsync(v, s);
    }
};

}  // namespace

static std::atomic<long long> g_launches{0};
void lu_count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

cudaError_t lu_sm_count(int *sms) {
    static std::atomic<int> cache[kMaxDev];
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kMaxDev) return cudaErrorInvalidDevice;
    int v = cache[d].load(std::memory_order_relaxed);
    if (v == 0) {
        if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d)) != cudaSuccess) return e;
        cache[d].store(v, std::memory_order_relaxed);
    }
    *sms = v;
    return cudaSuccess;
}

// trailing-update instrumentation (lu_update_timing)
namespace {
struct TimedLaunch {
    cudaEvent_t a, b;
    double flops, bytes;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<TimedLaunch> g_timed;

bool timing_on() {
    std::lock_guard<std::mutex> lk(g_tmu);
    return g_timing;
}

// launch trace of the factorization schedule (lu_trace)
struct TraceRec {
    int kind, step, stream;
    cudaEvent_t a, b;
};
bool g_trace_on = false;
std::vector<TraceRec> g_trace;

// per-CTA trace ring (lu_cta_trace), installed on one device
struct CtaRing {
    lu_cta_event *ring = nullptr;
    int *count = nullptr;
    int cap = 0;
    int dev = -1;
};
CtaRing g_cta;

// The trace argument for a launch of task `kind` at `step` (empty when off).
CtaTrace cta_tag(int kind, int step) {
    std::lock_guard<std::mutex> lk(g_tmu);
    CtaTrace t{nullptr, nullptr, 0, 0};
    int d = -1;
    if (g_cta.ring && cudaGetDevice(&d) == cudaSuccess && d == g_cta.dev) {
        t.ring = g_cta.ring;
        t.count = g_cta.count;
        t.cap = g_cta.cap;
        t.tag = (kind << 24) | (step & 0xffffff);
    }
    return t;
}

bool trace_on() {
    std::lock_guard<std::mutex> lk(g_tmu);
    return g_trace_on;
}

// Runs launch() on stream s; when tracing, brackets it with two events.
template <class F>
cudaError_t traced(int kind, int step, int sid, cudaStream_t s, F launch) {
    if (!trace_on()) return launch();
    TraceRec r{kind, step, sid, nullptr, nullptr};
    cudaError_t e;
    if ((e = cudaEventCreate(&r.a)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&r.b)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(r.a, s)) != cudaSuccess) return e;
    if ((e = launch()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(r.b, s)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tmu);
    g_trace.push_back(r);
    return cudaSuccess;
}
}  // namespace

void lu_note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_last_err, sizeof(g_last_err), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
    if (getenv("LU_DEBUG")) fprintf(stderr, "liblu: %s\n", g_last_err);
}

int *lu_device_status_ptr() {
    DevState *st = nullptr;
    if (dev_state(&st) != cudaSuccess) return nullptr;
    return st->status;
}

long long lu_spin_bound_ns(const lu_opts *o) {
    if (o && o->spin_ns > 0) return o->spin_ns;
    return 2000000000LL;
}

// ---------------------------------------------------------------------------
// blocked right-looking LU with look-ahead
// ---------------------------------------------------------------------------
namespace {

struct Plan {
    int bo = 0;       // outer panel width
    int bi = 0;       // inner panel width (cluster capacity)
    bool bi_auto = true;   // per panel: the widest inner width its row count allows
    bool tc = false;  // tensor-core update
    int fmt = 0;      // staging format: 0 BF16, 1 split BF16, 2 FP8 e4m3, 3 FP64 digit slices (StageDesc)
    int depth = 1;    // look-ahead depth d: strips k+1 .. k+d on the panel branch (0: none)
    int panel_ctas = 16;
    int update_ctas = 0;   // persistent CTAs of the remainder update (0: one per SM)
    bool share = true;     // worker sharing with the persistent tensor-core update (SmShare)
    int tile = 0;          // update tile shape (lu_opts.tile)
    int et = 0;            // early termination (lu_opts.early_term; look-ahead of depth 1 only)
    long long bound = 2000000000LL;
};

template <typename T>
Plan make_plan(int n, const lu_opts *o) {
    Plan p;
    const bool tc = (sizeof(T) == 4) && o &&
                    (o->update == LU_UPDATE_BF16 || o->update == LU_UPDATE_BF16X3 || o->update == LU_UPDATE_FP8);
    const bool emu = (sizeof(T) == 8) && o && o->update == LU_UPDATE_F64EMU;
    p.tc = tc || emu;
    p.fmt = emu ? 3 : (o && o->update == LU_UPDATE_BF16X3) ? 1 : ((o && o->update == LU_UPDATE_FP8) ? 2 : 0);
    if (emu) {
        // emulated FP64 update: K = b_o <= 64 (one 64-wide digit slice per operand row)
        p.bo = (o->nb > 0) ? std::min(o->nb, f64emu_kpad()) : f64emu_kpad();
    } else if (tc) {
        // the factorization is panel-bound up to n ~ 16k (the update is HBM-bound
        // with C traffic 8 n^3 / (3 b_o)): narrower panels keep the panel chain short
        p.bo = (o && o->nb > 0) ? o->nb : (n >= 24576 ? 128 : 64);
        p.bo = std::min(p.bo, tc_max_k());
    } else if (sizeof(T) == 4) {
        p.bo = (o && o->nb > 0) ? o->nb : 128;
    } else {
        // FP64: b_o = 32 up to n = 8192 and 64 beyond, inner panels as wide as the
        // cluster's register tiles hold (measured on GB300 at n = 32768: b_o = 8,
        // the inner width there, reaches 575 GFLOP/s; b_o = 64, 1221 GFLOP/s: a
        // narrow update streams C from HBM more often than the DFMA pipe needs)
        p.bo = (o && o->nb > 0) ? o->nb : (n >= 8192 ? 64 : 32);
    }
    const int bo_fit = std::min(std::max(p.bo, 1), 256);
    const int wfit = std::max(1, panel_width_that_fits(std::max(n, 1), sizeof(T), kPanelSmemCap, 64, p.bo > 0 ? bo_fit : 0));
    if (p.bo == 0) p.bo = std::min(32, wfit);
    p.bo = std::min(p.bo, 256);
    p.bi_auto = !(o && o->nb_inner > 0);
    p.bi = p.bi_auto ? wfit : std::min(o->nb_inner, wfit);
    p.bi = std::max(1, std::min(p.bi, p.bo));
    p.depth = (o && o->lookahead < 0) ? 0 : ((o && o->lookahead > 1) ? std::min(o->lookahead, kMaxDepth) : 1);
    // FP64 panels: an 8-CTA team by default (the autotuner's choice at n = 512 ... 16384);
    // the geometry takes more CTAs when the rows do not fit 8
    p.panel_ctas = (o && o->panel_ctas > 0) ? std::min(16, o->panel_ctas) : (sizeof(T) == 8 ? 8 : 16);
    p.update_ctas = (o && o->update_ctas > 0) ? o->update_ctas : 0;
    p.share = !(o && o->sm_share < 0);
    p.tile = o ? o->tile : 0;
    p.et = (o && p.depth == 1) ? o->early_term : 0;
    p.bound = lu_spin_bound_ns(o);
    return p;
}

// Options with every field left at zero filled from the autotuner's table
// entry for (kind, dt, update, n), when it has one.
const lu_opts *with_tuned(int kind, lu_dtype dt, int n, const lu_opts *o, lu_opts *buf) {
    lu_opts t;
    if (!lu_tune_get(kind, dt, o ? o->update : LU_UPDATE_NATIVE, n, &t)) return o;
    *buf = o ? *o : lu_opts{};
    if (buf->nb == 0) buf->nb = t.nb;
    if (buf->nb_inner == 0) buf->nb_inner = t.nb_inner;
    if (buf->panel_ctas == 0) buf->panel_ctas = t.panel_ctas;
    if (buf->lookahead == 0) buf->lookahead = t.lookahead;
    if (buf->update_ctas == 0) buf->update_ctas = t.update_ctas;
    if (buf->tile == 0) buf->tile = t.tile;
    return buf;
}

template <typename T>
struct FactorCtx {
    int n;
    T *A;
    int lda;
    int *ipiv;
    int *info;
    int *perm;            // optional
    Plan pl;
    DevState *st;
    int ring = 2;         // panels in flight: look-ahead depth + 1 (2 at least)
    int *maps[kRing] = {};                        // row maps of panels k (slot k % ring)
    unsigned char *stA[kRing] = {};               // staged L21 of panels k (slot k % ring), bytes
    unsigned char *stB = nullptr;                 // staged U12
    float *scA[kRing] = {};                       // FP8: row scales of stA
    float *scB = nullptr;                         // FP8: column scales of stB
    double *dscA[kRing] = {};                     // FP64 digit slices: row scales of stA
    double *dscB = nullptr;                       // FP64 digit slices: column scales of stB
    int kpad = 0;
    int kinner = 0;   // staged elements per row/column (kpad, or 2 kpad when split)
    CUtensorMap mapA[kRing], mapB;
    int *tile_ctr = nullptr;   // [0]: panel-branch updates, [1]: remainder-branch updates
};

template <typename T>
cudaError_t update_launch(FactorCtx<T> &c, int k_par, int kb, int w, int c0, int c1, cudaStream_t s, CtaTrace tr,
                          SmShare sh);

// C[rows r0.., cols c0..c1) -= L(rows r0.., cols kb..kb+w) * U(rows kb..kb+w, cols c0..c1)
// sh: worker sharing of a persistent tensor-core update (SmShare; ignored by the SIMT update)
template <typename T>
cudaError_t update(FactorCtx<T> &c, int k_par, int kb, int w, int c0, int c1, cudaStream_t s, CtaTrace tr,
                   SmShare sh = SmShare{}) {
    const int r0 = kb + w;
    const int m = c.n - r0, nn = c1 - c0;
    if (m <= 0 || nn <= 0) return cudaSuccess;
    if (!timing_on() || sh.mode == 1) return update_launch<T>(c, k_par, kb, w, c0, c1, s, tr, sh);
    TimedLaunch t;
    cudaError_t e;
    if ((e = cudaEventCreate(&t.a)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&t.b)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(t.a, s)) != cudaSuccess) return e;
    if ((e = update_launch<T>(c, k_par, kb, w, c0, c1, s, tr, sh)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(t.b, s)) != cudaSuccess) return e;
    const int k = c.pl.tc ? c.kinner : w;   // staged operand width (hi and lo halves with the split)
    const double opw = c.pl.tc ? (c.pl.fmt == 2 ? 1.0 : 2.0) : (double)sizeof(T);
    t.flops = 2.0 * m * nn * (double)w;
    t.bytes = 2.0 * m * nn * sizeof(T) + (double)m * k * opw + (double)k * nn * opw;
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timed.push_back(t);
    return cudaSuccess;
}

template <typename T>
cudaError_t update_launch(FactorCtx<T> &c, int k_par, int kb, int w, int c0, int c1, cudaStream_t s, CtaTrace tr,
                          SmShare sh) {
    const int r0 = kb + w;
    const int m = c.n - r0, nn = c1 - c0;
    // task counters: [0] the panel branch's updates, [1] the remainder update and its joiners
    const bool ru = s != c.st->P;
    if constexpr (sizeof(T) == 8) {
        if (c.pl.tc)
            return launch_gemm_f64emu(m, nn, c.mapA[k_par], 0, c.mapB, c0 - r0, reinterpret_cast<double *>(c.A) + r0 + (size_t)c0 * c.lda,
                                      c.lda, c.dscA[k_par], c.dscB, c.tile_ctr + (ru ? 1 : 0), c.st->status,
                                      c.pl.bound, ru ? c.pl.update_ctas : 0, s, tr, -1, sh, c.pl.tile);
    }
    if constexpr (sizeof(T) == 4) {
        if (c.pl.tc)
            return launch_gemm_tc(c.pl.fmt == 1 ? 3 : (c.pl.fmt == 2 ? 8 : 1), m, nn, c.kpad, c.mapA[k_par], 0, c.mapB,
                                  c0 - r0, reinterpret_cast<float *>(c.A) + r0 + (size_t)c0 * c.lda, c.lda,
                                  c.tile_ctr + (ru ? 1 : 0), c.st->status, c.pl.bound, s, c.scA[k_par], c.scB,
                                  ru ? c.pl.update_ctas : 0, tr, sh);
    }
    return launch_gemm_simt<T>(m, nn, w, c.A + r0 + (size_t)kb * c.lda, c.lda, c.A + kb + (size_t)c0 * c.lda, c.lda,
                               c.A + r0 + (size_t)c0 * c.lda, c.lda, s, tr, false, -1, c.pl.tile);
}

template <typename T>
cudaError_t swap_trsm(FactorCtx<T> &c, int kb, int w, const int *map, int c0, int c1, int do_trsm, cudaStream_t s,
                      CtaTrace tr) {
    StageDesc sd{nullptr, nullptr, c.kinner, c.kpad, c.pl.fmt, nullptr};
    if (do_trsm && c.pl.tc) { sd.ptr = c.stB; sd.scale = c.scB; sd.dscale = c.dscB; }
    return launch_swap_trsm<T>(c.A, c.lda, kb, w, map, c0, c1, do_trsm, sd, kb + w, s, tr);
}

// Inner width of the outer panel at column kb (width w) of an order-n
// factorization: the panel's rows shrink with k, so later panels hold wider
// inner panels.
int plan_inner_width(const Plan &pl, int n, size_t elem, int kb, int w) {
    int bi = pl.bi;
    if (pl.bi_auto) bi = std::max(bi, panel_width_that_fits(n - kb, elem, kPanelSmemCap, 64, w));
    return std::min(bi, w);
}

// Whether every outer panel of the plan fits a cluster (with early termination
// a panel may start at any column).
bool plan_fits(const Plan &pl, int n, size_t elem) {
    for (int kb = 0; kb < n; kb += pl.et ? 1 : pl.bo) {
        const int w = std::min(pl.bo, n - kb);
        if (!panel_fits(n - kb, elem, w, plan_inner_width(pl, n, elem, kb, w), pl.panel_ctas, kPanelSmemCap)) return false;
    }
    return true;
}

// Factor outer panel at column kb (width w) on stream s: one cluster launch
// that also leaves the row map in maps[par], updates perm and stages L21.
template <typename T>
cudaError_t factor_outer_panel(FactorCtx<T> &c, int kb, int w, int par, cudaStream_t s, CtaTrace tr, int *yreq = nullptr,
                               EtArgs et = EtArgs{}) {
    StageDesc sd{nullptr, nullptr, c.kinner, c.kpad, c.pl.fmt, nullptr};
    if (c.pl.tc && kb + w < c.n) { sd.ptr = c.stA[par]; sd.scale = c.scA[par]; sd.dscale = c.dscA[par]; }
    return launch_panel_outer<T>(c.A + kb + (size_t)kb * c.lda, c.lda, c.n - kb, w, plan_inner_width(c.pl, c.n, sizeof(T), kb, w),
                                 c.ipiv + kb, kb,
                                 c.info, c.maps[par], c.perm, sd, c.pl.panel_ctas, kPanelSmemCap, c.st->status,
                                 c.pl.bound, s, tr, yreq, et);
}

// The SMs of one placement of a C-CTA panel cluster (SmShare), found by a probe
// cluster on stream s the first time C is asked for; nullptr where the probe
// launch was refused.
const unsigned *share_mask_for(DevState *st, int C, cudaStream_t s) {
    if (C < 1 || C > 16 || st->sms > (int)kShareMaskBits) return nullptr;
    unsigned *mask = st->share_mask + (size_t)C * kMaskWords;
    if (st->share_state[C] == 0) {
        st->share_state[C] = -1;
        if (cudaMemsetAsync(mask, 0, kMaskWords * sizeof(unsigned), s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (launch_cluster_sm_probe(C, mask, s) != cudaSuccess) {
            cudaGetLastError();   // cluster size refused: no sharing at this size
            return nullptr;
        }
        st->share_state[C] = 1;
    }
    return st->share_state[C] > 0 ? mask : nullptr;
}

template <typename T>
int factor_core(int n, T *A, int lda, int *ipiv, int *info, int *perm, const Plan &pl, cudaStream_t caller);

template <typename T>
int factor_impl(int n, T *A, int lda, int *ipiv, int *info, int *perm, const Plan &pl, cudaStream_t caller) {
    LU_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), caller));
    if (n == 0) return LU_OK;
    if (pl.tc && sizeof(T) == 4 && !(((uintptr_t)A % 16 == 0) && lda % 4 == 0)) {
        // the tensor-core update moves C with TMA (16-byte aligned columns):
        // factor an aligned copy and copy the factors back
        Workspace ws(caller);
        const int ld2 = (n + 3) & ~3;
        T *A2 = nullptr;
        LU_CUDA_TRY(ws.get(&A2, (size_t)ld2 * n));
        LU_CUDA_TRY(cudaMemcpy2DAsync(A2, sizeof(T) * ld2, A, sizeof(T) * lda, sizeof(T) * n, n, cudaMemcpyDeviceToDevice, caller));
        int rc = factor_core<T>(n, A2, ld2, ipiv, info, perm, pl, caller);
        if (rc != LU_OK) return rc;
        LU_CUDA_TRY(cudaMemcpy2DAsync(A, sizeof(T) * lda, A2, sizeof(T) * ld2, sizeof(T) * n, n, cudaMemcpyDeviceToDevice, caller));
        return LU_OK;
    }
    return factor_core<T>(n, A, lda, ipiv, info, perm, pl, caller);
}

template <typename T>
int factor_core(int n, T *A, int lda, int *ipiv, int *info, int *perm, const Plan &pl, cudaStream_t caller) {
    DevState *st = nullptr;
    LU_CUDA_TRY(dev_state(&st));
    std::lock_guard<std::recursive_mutex> lk(g_enqueue_mu);
    // early termination (section 4.2): the host learns each panel's width before it
    // enqueues the next step, which a stream under capture cannot give
    const bool et = pl.et != 0 && pl.depth == 1;
    if (et) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        LU_CUDA_TRY(cudaStreamIsCapturing(caller, &cs));
        if (cs != cudaStreamCaptureStatusNone) return LU_ERR_UNSUPPORTED;
    }
    Workspace ws(caller);
    FactorCtx<T> c;
    c.n = n; c.A = A; c.lda = lda; c.ipiv = ipiv; c.info = info; c.perm = perm; c.pl = pl; c.st = st;
    const int bo = pl.bo;
    // every panel of the plan must fit a cluster before anything is enqueued
    if (!plan_fits(pl, n, sizeof(T))) return LU_ERR_UNSUPPORTED;
    st->widths.clear();
    st->widths_valid = false;
    c.ring = std::max(2, pl.depth + 1);
    for (int i = 0; i < c.ring; ++i) LU_CUDA_TRY(ws.get(&c.maps[i], (size_t)(1 + 4 * bo)));
    LU_CUDA_TRY(ws.get(&c.tile_ctr, 2));
    if (perm) LU_CUDA_TRY(launch_iota(perm, n, caller));
    if (pl.tc && pl.fmt == 3) {
        // FP64 digit slices: kF64Slices slices of 64 K-elements per staged row / column
        c.kpad = f64emu_kpad();
        c.kinner = c.kpad * kF64Slices;
        for (int i = 0; i < c.ring; ++i) {
            LU_CUDA_TRY(ws.get(&c.stA[i], (size_t)n * c.kinner * 2));
            LU_CUDA_TRY(ws.get(&c.dscA[i], (size_t)n));
            LU_CUDA_TRY(make_stage_map(&c.mapA[i], c.stA[i], c.kinner, n, c.kinner, f64emu_box_rows(), 0));
        }
        LU_CUDA_TRY(ws.get(&c.stB, (size_t)n * c.kinner * 2));
        LU_CUDA_TRY(ws.get(&c.dscB, (size_t)n));
        LU_CUDA_TRY(make_stage_map(&c.mapB, c.stB, c.kinner, n, c.kinner, f64emu_box_cols(), 0));
    } else if (pl.tc) {
        const int fp8 = pl.fmt == 2;
        c.kpad = tc_kpad(bo, fp8);
        c.kinner = c.kpad * (pl.fmt == 1 ? 2 : 1);
        const size_t esz = fp8 ? 1 : 2;
        for (int i = 0; i < c.ring; ++i) LU_CUDA_TRY(ws.get(&c.stA[i], (size_t)n * c.kinner * esz));
        LU_CUDA_TRY(ws.get(&c.stB, (size_t)n * c.kinner * esz));
        if (fp8) {
            for (int i = 0; i < c.ring; ++i) LU_CUDA_TRY(ws.get(&c.scA[i], (size_t)n));
            LU_CUDA_TRY(ws.get(&c.scB, (size_t)n));
        }
        for (int i = 0; i < c.ring; ++i)
            LU_CUDA_TRY(make_stage_map(&c.mapA[i], c.stA[i], c.kinner, n, c.kinner, tc_box_rows(), fp8));
        LU_CUDA_TRY(make_stage_map(&c.mapB, c.stB, c.kinner, n, c.kinner, tc_box_cols(), fp8));
    }
    cudaStream_t P = st->P, U = st->U;
    if (et) LU_CUDA_TRY(cudaMemsetAsync(st->et, 0, 2 * sizeof(int), caller));
    LU_CUDA_TRY(cudaEventRecord(st->evIn, caller));
    LU_CUDA_TRY(cudaStreamWaitEvent(P, st->evIn, 0));
    LU_CUDA_TRY(cudaStreamWaitEvent(U, st->evIn, 0));

    const int depth = pl.depth, R = c.ring;
    // prologue: panel 0
    LU_CUDA_TRY(traced(LU_TRACE_PANEL, 0, 0, P,
                       [&] { return factor_outer_panel<T>(c, 0, std::min(bo, n), 0, P, cta_tag(LU_TRACE_PANEL, 0)); }));
    LU_CUDA_TRY(cudaEventRecord(st->evP[0], P));
    // panel k starts at column kb with nominal width wnom and factored w columns
    // (w < wnom only after an early termination)
    int kb = 0, wnom = std::min(bo, n), w = wnom;
    for (int k = 0; kb < n; ++k) {
        const int sl = k % R, sl1 = (k + 1) % R, slp = (k + R - 1) % R;
        const int cn0 = kb + w, wn = std::min(bo, n - cn0);
        // columns [cn0, kb + wnom) are those an early-terminated panel k left: the panel
        // already gave them step k (interchanges, U12 rows, update), so strip k+1 takes
        // step k only from column kb + wnom on
        const int fresh0 = std::min(std::max(cn0, kb + wnom), cn0 + wn);
        const int *map = c.maps[sl];
        // look-ahead window: strips k+1 .. k+depth on the panel branch, the rest on RU
        const int rest0 = std::min(n, cn0 + depth * bo);
        // worker sharing with a persistent remainder update (SmShare): the SMs of one
        // placement of panel k+1's cluster
        const unsigned *smask = nullptr;
        int cctas = 0;
        if (pl.tc && pl.share && depth > 0 && wn > 0 && rest0 < n) {
            cctas = panel_cluster_ctas(n - cn0, sizeof(T), wn, plan_inner_width(pl, n, sizeof(T), cn0, wn), pl.panel_ctas,
                                       kPanelSmemCap);
            smask = share_mask_for(st, cctas, P);
        }
        // ---- T_RU on U, first part: interchanges left of panel k, RU1 ------------
        LU_CUDA_TRY(cudaStreamWaitEvent(U, st->evP[sl], 0));
        if (kb > 0)
            LU_CUDA_TRY(traced(LU_TRACE_SWAP_LEFT, k, 1, U,
                               [&] { return swap_trsm<T>(c, kb, w, map, 0, kb, 0, U, cta_tag(LU_TRACE_SWAP_LEFT, k)); }));
        if (rest0 < n)
            LU_CUDA_TRY(traced(LU_TRACE_RU1, k, 1, U,
                               [&] { return swap_trsm<T>(c, kb, w, map, rest0, n, 1, U, cta_tag(LU_TRACE_RU1, k)); }));
        // ---- T_PF on P: PF1, PF2 on strip k+1, then PF3 = panel k+1 ------------------
        if (wn > 0 && depth > 0) {
            // strip k+1 was last updated by RU2(k-1) with depth 1, by this branch with depth >= 2
            if (k > 0 && depth == 1) LU_CUDA_TRY(cudaStreamWaitEvent(P, st->evU[slp], 0));
            if (fresh0 < cn0 + wn) {
                LU_CUDA_TRY(traced(LU_TRACE_PF1, k, 0, P, [&] {
                    return swap_trsm<T>(c, kb, w, map, fresh0, cn0 + wn, 1, P, cta_tag(LU_TRACE_PF1, k));
                }));
                LU_CUDA_TRY(traced(LU_TRACE_PF2, k, 0, P,
                                   [&] { return update<T>(c, sl, kb, w, fresh0, cn0 + wn, P, cta_tag(LU_TRACE_PF2, k)); }));
            }
            // RU2 starts after PF2: when both become ready the panel (higher
            // priority) is dispatched first, and RU2's queued CTAs fill the
            // rest of the GPU and later the SMs the panel cluster frees
            LU_CUDA_TRY(cudaEventRecord(st->evPF2, P));
            // with a persistent RU2 that may already hold every SM: ask one cluster
            // placement back; the panel withdraws the request once it runs
            if (smask) LU_CUDA_TRY(launch_share_raise(st->share_req, P));
            // early termination: panel k+1 stops at the end of the inner panel during
            // which RU2(k) (below, on U) raised the flag to k + 1
            const EtArgs eta = et ? EtArgs{st->et, k + 1, pl.et == 2 ? 1 : 0, st->et + 1} : EtArgs{};
            LU_CUDA_TRY(traced(LU_TRACE_PANEL, k + 1, 0, P, [&] {
                return factor_outer_panel<T>(c, cn0, wn, sl1, P, cta_tag(LU_TRACE_PANEL, k + 1),
                                             smask ? st->share_req : nullptr, eta);
            }));
            if (smask) LU_CUDA_TRY(cudaEventRecord(st->evPanelEnd, P));
            // depth >= 2: strips k+2 .. k+depth after the panel, off its chain; the last of
            // them was in RU2(k-1)'s range
            const int s0 = cn0 + wn;
            if (s0 < rest0) {
                if (k > 0) LU_CUDA_TRY(cudaStreamWaitEvent(P, st->evU[slp], 0));
                LU_CUDA_TRY(traced(LU_TRACE_PF1, k, 0, P,
                                   [&] { return swap_trsm<T>(c, kb, w, map, s0, rest0, 1, P, cta_tag(LU_TRACE_PF1, k)); }));
                LU_CUDA_TRY(traced(LU_TRACE_PF2, k, 0, P,
                                   [&] { return update<T>(c, sl, kb, w, s0, rest0, P, cta_tag(LU_TRACE_PF2, k)); }));
            }
            // the remainder branch of step k+1 starts after this branch's step k: its first
            // task applies panel k+1's interchanges to the columns left of it, rows of
            // L21(k) included, which the strip updates above read
            LU_CUDA_TRY(cudaEventRecord(st->evP[sl1], P));
            LU_CUDA_TRY(cudaStreamWaitEvent(U, st->evPF2, 0));
        }
        // ---- T_RU on U, second part: RU2 ----------------------------------------------
        if (rest0 < n && smask) {
            // RU2's CTAs on the requested SMs stop at a task boundary while the request
            // stands; a grid of the panel's size joins RU2's task queue on J when the
            // panel ends (the PF team joining RU2, section 4.1), and RU2 counts as done
            // when both have drained the queue
            LU_CUDA_TRY(cudaMemsetAsync(c.tile_ctr + 1, 0, sizeof(int), U));
            LU_CUDA_TRY(cudaEventRecord(st->evGo, U));
            const SmShare sh{st->share_req, smask, 2, 0};
            LU_CUDA_TRY(traced(LU_TRACE_RU2, k, 1, U,
                               [&] { return update<T>(c, sl, kb, w, rest0, n, U, cta_tag(LU_TRACE_RU2, k), sh); }));
            LU_CUDA_TRY(cudaStreamWaitEvent(st->J, st->evPanelEnd, 0));
            LU_CUDA_TRY(cudaStreamWaitEvent(st->J, st->evGo, 0));
            LU_CUDA_TRY(update<T>(c, sl, kb, w, rest0, n, st->J, cta_tag(LU_TRACE_RU2, k), SmShare{nullptr, nullptr, 1, cctas}));
            LU_CUDA_TRY(cudaEventRecord(st->evJ, st->J));
            LU_CUDA_TRY(cudaStreamWaitEvent(U, st->evJ, 0));
        } else if (rest0 < n) {
            LU_CUDA_TRY(traced(LU_TRACE_RU2, k, 1, U,
                               [&] { return update<T>(c, sl, kb, w, rest0, n, U, cta_tag(LU_TRACE_RU2, k)); }));
        }
        if (et) LU_CUDA_TRY(launch_et_signal(st->et, k + 1, U));   // RU2(k) is done
        LU_CUDA_TRY(cudaEventRecord(st->evU[sl], U));
        if (wn > 0 && depth == 0) {
            LU_CUDA_TRY(cudaStreamWaitEvent(P, st->evU[sl], 0));
            LU_CUDA_TRY(traced(LU_TRACE_PANEL, k + 1, 0, P,
                               [&] { return factor_outer_panel<T>(c, cn0, wn, sl1, P, cta_tag(LU_TRACE_PANEL, k + 1)); }));
            LU_CUDA_TRY(cudaEventRecord(st->evP[sl1], P));
        }
        st->widths.push_back(w);
        // the next step: panel k+1's width, read back once the panel has run
        int wnext = wn;
        if (et && wn > 0) {
            int hw = 0;
            LU_CUDA_TRY(cudaMemcpyAsync(&hw, st->et + 1, sizeof(int), cudaMemcpyDeviceToHost, P));
            LU_CUDA_TRY(cudaStreamSynchronize(P));
            if (hw < 1 || hw > wn) return LU_ERR_CUDA;   // the panel reports a width in [1, wn]
            wnext = hw;
        }
        kb = cn0;
        wnom = wn;
        w = wnext;
    }
    st->widths_valid = true;
    LU_CUDA_TRY(cudaEventRecord(st->evOutP, P));
    LU_CUDA_TRY(cudaEventRecord(st->evOutU, U));
    LU_CUDA_TRY(cudaStreamWaitEvent(caller, st->evOutP, 0));
    LU_CUDA_TRY(cudaStreamWaitEvent(caller, st->evOutU, 0));
    LU_CUDA_TRY(cudaGetLastError());
    return LU_OK;
}

template <typename T>
int solve_impl(int n, int nrhs, const T *LU, int lda, const int *ipiv, const int *perm_opt, T *B, int ldb, long long bound,
               cudaStream_t s, const T *Dinv = nullptr) {
    DevState *st = nullptr;
    LU_CUDA_TRY(dev_state(&st));
    if (n == 0 || nrhs == 0) return LU_OK;
    Workspace ws(s);
    int *perm = const_cast<int *>(perm_opt);
    if (!perm) {
        LU_CUDA_TRY(ws.get(&perm, n));
        LU_CUDA_TRY(launch_ipiv_to_perm(ipiv, n, perm, s));
    }
    T *X = nullptr;
    LU_CUDA_TRY(ws.get(&X, (size_t)n * nrhs));
    LU_CUDA_TRY((launch_gather_rows<T, T>(n, nrhs, perm, B, ldb, X, n, s)));
    int *tws = nullptr;
    LU_CUDA_TRY(ws.get(&tws, trsv_workspace_ints(n, nrhs)));
    LU_CUDA_TRY(launch_trsv_pair<T>(LU, lda, n, nrhs, X, n, tws, st->status, bound, st->sms, s, Dinv));
    LU_CUDA_TRY(cudaMemcpy2DAsync(B, sizeof(T) * ldb, X, sizeof(T) * n, sizeof(T) * n, nrhs, cudaMemcpyDeviceToDevice, s));
    return LU_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

static bool opts_valid(lu_dtype dt, const lu_opts *opts) {
    if (!opts) return true;
    if (opts->nb < 0 || opts->nb_inner < 0 || opts->panel_ctas < 0 || opts->panel_ctas > 16 || opts->update_ctas < 0 ||
        opts->sm_share < -1 || opts->sm_share > 1 || opts->tile < 0 || opts->tile > 2 || opts->early_term < 0 ||
        opts->early_term > 2 || (opts->early_term != 0 && (opts->lookahead < 0 || opts->lookahead > 1)) ||
        (opts->update != LU_UPDATE_NATIVE && opts->update != LU_UPDATE_BF16 && opts->update != LU_UPDATE_BF16X3 &&
         opts->update != LU_UPDATE_FP8 && opts->update != LU_UPDATE_F64EMU))
        return false;
    if (opts->update == LU_UPDATE_F64EMU) return dt == LU_F64 && opts->nb <= f64emu_kpad();
    if (opts->update != LU_UPDATE_NATIVE && dt != LU_F32) return false;
    if (opts->update != LU_UPDATE_NATIVE && opts->nb > tc_max_k()) return false;
    return true;
}

int lu_plan_info(lu_dtype dt, int n, const lu_opts *opts, lu_opts *plan) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (n < 1) return -2;
    if (!opts_valid(dt, opts)) return -3;
    if (!plan) return -4;
    lu_opts tuned;
    opts = with_tuned(0, dt, n, opts, &tuned);
    const Plan p = dt == LU_F64 ? make_plan<double>(n, opts) : make_plan<float>(n, opts);
    const size_t elem = dt == LU_F64 ? 8 : 4;
    *plan = lu_opts{};
    plan->nb = p.bo;
    plan->nb_inner = plan_inner_width(p, n, elem, 0, std::min(p.bo, n));
    plan->panel_ctas = p.panel_ctas;
    plan->lookahead = p.depth > 0 ? p.depth : -1;
    plan->update = opts ? opts->update : LU_UPDATE_NATIVE;
    plan->spin_ns = p.bound;
    plan->update_ctas = p.update_ctas;
    plan->sm_share = p.share ? 1 : -1;
    plan->tile = p.tile;
    plan->early_term = p.et;
    return plan_fits(p, n, elem) ? LU_OK : LU_ERR_UNSUPPORTED;
}

int lu_last_panel_widths(int *widths, int cap) {
    DevState *st = nullptr;
    if (dev_state(&st) != cudaSuccess) return -1;
    std::lock_guard<std::recursive_mutex> lk(g_enqueue_mu);
    if (!st->widths_valid) return -1;
    const int cnt = (int)st->widths.size();
    if (widths)
        for (int i = 0; i < std::min(cnt, cap); ++i) widths[i] = st->widths[i];
    return cnt;
}

int lu_factor(lu_dtype dt, int n, void *dA, int lda, int *d_ipiv, int *d_info, const lu_opts *opts, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (n < 0) return -2;
    if (n > 0 && !dA) return -3;
    if (lda < std::max(1, n)) return -4;
    if (n > 0 && !d_ipiv) return -5;
    if (!d_info) return -6;
    if (!opts_valid(dt, opts)) return -7;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lu_opts tuned;
    opts = with_tuned(0, dt, n, opts, &tuned);
    if (dt == LU_F64) {
        Plan p = make_plan<double>(n, opts);
        return factor_impl<double>(n, static_cast<double *>(dA), lda, d_ipiv, d_info, nullptr, p, s);
    }
    Plan p = make_plan<float>(n, opts);
    return factor_impl<float>(n, static_cast<float *>(dA), lda, d_ipiv, d_info, nullptr, p, s);
}

int lu_solve(lu_dtype dt, int n, int nrhs, const void *dLU, int lda, const int *d_ipiv, void *dB, int ldb, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (n > 0 && !dLU) return -4;
    if (lda < std::max(1, n)) return -5;
    if (n > 0 && !d_ipiv) return -6;
    if (n > 0 && nrhs > 0 && !dB) return -7;
    if (ldb < std::max(1, n)) return -8;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dt == LU_F64)
        return solve_impl<double>(n, nrhs, static_cast<const double *>(dLU), lda, d_ipiv, nullptr, static_cast<double *>(dB),
                                  ldb, lu_spin_bound_ns(nullptr), s);
    return solve_impl<float>(n, nrhs, static_cast<const float *>(dLU), lda, d_ipiv, nullptr, static_cast<float *>(dB), ldb,
                             lu_spin_bound_ns(nullptr), s);
}

int lu_factor_batched(lu_dtype dt, int batch, const int *d_n, void *const *d_A, const int *d_lda, int *const *d_ipiv,
                      int *d_info, int max_n, const lu_opts *opts, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (batch < 0) return -2;
    if (batch > 0 && !d_n) return -3;
    if (batch > 0 && !d_A) return -4;
    if (batch > 0 && !d_lda) return -5;
    if (batch > 0 && !d_ipiv) return -6;
    if (batch > 0 && !d_info) return -7;
    if (max_n < 0 || max_n > 1024) return -8;
    if (batch > 2147483647 / 2) return -2;
    int nb = opts ? opts->nb : 0;
    if (nb != 0 && nb != 1 && nb != 16 && nb != 32) return -9;
    lu_opts tuned;
    if (nb == 0 && lu_tune_get(1, dt, LU_UPDATE_NATIVE, max_n, &tuned) && (tuned.nb <= 1 || max_n <= kBatchedBlockedMaxN))
        nb = tuned.nb;
    if ((nb == 16 || nb == 32) && max_n > kBatchedBlockedMaxN) return -9;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nb == 1 || max_n > kBatchedBlockedMaxN) {
        // the unblocked kernel: one CTA per matrix, the algorithm of Figure 1 (left) as written
        if (dt == LU_F64)
            LU_CUDA_TRY(launch_getrf_batched<double>(batch, d_n, reinterpret_cast<double *const *>(d_A), d_lda, d_ipiv, d_info, max_n, s));
        else
            LU_CUDA_TRY(launch_getrf_batched<float>(batch, d_n, reinterpret_cast<float *const *>(d_A), d_lda, d_ipiv, d_info, max_n, s));
        return LU_OK;
    }
    if (batch == 0) return LU_OK;
    DevState *st = nullptr;
    LU_CUDA_TRY(dev_state(&st));
    Workspace ws(s);
    int *bws = nullptr;
    LU_CUDA_TRY(ws.get(&bws, batched_blocked_workspace_ints(batch)));
    if (dt == LU_F64)
        LU_CUDA_TRY(launch_getrf_batched_blocked<double>(batch, d_n, reinterpret_cast<double *const *>(d_A), d_lda, d_ipiv,
                                                         d_info, nb, bws, st->sms, s));
    else
        LU_CUDA_TRY(launch_getrf_batched_blocked<float>(batch, d_n, reinterpret_cast<float *const *>(d_A), d_lda, d_ipiv,
                                                        d_info, nb, bws, st->sms, s));
    return LU_OK;
}

int lu_solve_batched(lu_dtype dt, int batch, int nrhs, const int *d_n, const void *const *d_LU, const int *d_lda,
                     const int *const *d_ipiv, void *const *d_B, const int *d_ldb, int max_n, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (batch < 0) return -2;
    if (nrhs < 0) return -3;
    if (batch > 0 && !d_n) return -4;
    if (batch > 0 && !d_LU) return -5;
    if (batch > 0 && !d_lda) return -6;
    if (batch > 0 && !d_ipiv) return -7;
    if (batch > 0 && !d_B) return -8;
    if (batch > 0 && !d_ldb) return -9;
    if (max_n < 0 || max_n > 1024) return -10;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (max_n <= kBatchedBlockedMaxN) {
        // one warp per (matrix, right-hand side)
        DevState *st = nullptr;
        LU_CUDA_TRY(dev_state(&st));
        if (dt == LU_F64)
            LU_CUDA_TRY(launch_getrs_batched_warp<double>(batch, nrhs, d_n, reinterpret_cast<const double *const *>(d_LU),
                                                          d_lda, d_ipiv, reinterpret_cast<double *const *>(d_B), d_ldb,
                                                          st->sms, s));
        else
            LU_CUDA_TRY(launch_getrs_batched_warp<float>(batch, nrhs, d_n, reinterpret_cast<const float *const *>(d_LU),
                                                         d_lda, d_ipiv, reinterpret_cast<float *const *>(d_B), d_ldb,
                                                         st->sms, s));
        return LU_OK;
    }
    if (dt == LU_F64)
        LU_CUDA_TRY(launch_getrs_batched<double>(batch, nrhs, d_n, reinterpret_cast<const double *const *>(d_LU), d_lda, d_ipiv,
                                                 reinterpret_cast<double *const *>(d_B), d_ldb, max_n, s));
    else
        LU_CUDA_TRY(launch_getrs_batched<float>(batch, nrhs, d_n, reinterpret_cast<const float *const *>(d_LU), d_lda, d_ipiv,
                                                reinterpret_cast<float *const *>(d_B), d_ldb, max_n, s));
    return LU_OK;
}

int lu_trailing_update(int update, int m, int n, int k, const float *dA, int lda, const float *dB, int ldb, float *dC,
                       int ldc, void *stream) {
    if (update != LU_UPDATE_NATIVE && update != LU_UPDATE_BF16 && update != LU_UPDATE_BF16X3 && update != LU_UPDATE_FP8)
        return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (k < 0 || (update != LU_UPDATE_NATIVE && k > tc_max_k())) return -4;
    if (m > 0 && k > 0 && !dA) return -5;
    if (lda < std::max(1, m)) return -6;
    if (n > 0 && k > 0 && !dB) return -7;
    if (ldb < std::max(1, k)) return -8;
    if (m > 0 && n > 0 && !dC) return -9;
    if (ldc < std::max(1, m)) return -10;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (m == 0 || n == 0 || k == 0) return LU_OK;
    if (update == LU_UPDATE_NATIVE) {
        LU_CUDA_TRY(launch_gemm_simt<float>(m, n, k, dA, lda, dB, ldb, dC, ldc, s));
        return LU_OK;
    }
    DevState *st = nullptr;
    LU_CUDA_TRY(dev_state(&st));
    Workspace ws(s);
    const int fp8 = update == LU_UPDATE_FP8;
    const int kpad = tc_kpad(k, fp8);
    const int split = update == LU_UPDATE_BF16X3;
    const int kinner = kpad * (split ? 2 : 1);
    const int nprod = fp8 ? 8 : (split ? 3 : 1);
    void *sa = nullptr, *sb = nullptr;
    float *scA = nullptr, *scB = nullptr;
    if (fp8) {
        unsigned char *a8 = nullptr, *b8 = nullptr;
        LU_CUDA_TRY(ws.get(&a8, (size_t)m * kinner));
        LU_CUDA_TRY(ws.get(&b8, (size_t)n * kinner));
        LU_CUDA_TRY(ws.get(&scA, (size_t)m));
        LU_CUDA_TRY(ws.get(&scB, (size_t)n));
        LU_CUDA_TRY(launch_stage_rows_fp8(m, k, kpad, dA, lda, a8, kinner, scA, s));
        LU_CUDA_TRY(launch_stage_cols_fp8(k, kpad, n, dB, ldb, b8, kinner, scB, s));
        sa = a8;
        sb = b8;
    } else {
        __nv_bfloat16 *a16 = nullptr, *b16 = nullptr;
        LU_CUDA_TRY(ws.get(&a16, (size_t)m * kinner));
        LU_CUDA_TRY(ws.get(&b16, (size_t)n * kinner));
        LU_CUDA_TRY(launch_stage_rows(m, k, kpad, dA, lda, a16, kinner, split, s));
        LU_CUDA_TRY(launch_stage_cols(k, kpad, n, dB, ldb, b16, kinner, split, s));
        sa = a16;
        sb = b16;
    }
    CUtensorMap ma, mb;
    int *ctr = nullptr;
    LU_CUDA_TRY(ws.get(&ctr, 1));
    LU_CUDA_TRY(make_stage_maps(&ma, sa, m, &mb, sb, n, kinner, kinner, fp8));
    if (tc_c_aligned(dC, ldc)) {
        LU_CUDA_TRY(launch_gemm_tc(nprod, m, n, kpad, ma, 0, mb, 0, dC, ldc, ctr, st->status, lu_spin_bound_ns(nullptr), s,
                                   scA, scB));
    } else {
        // the kernel moves C with TMA (16-byte aligned rows): work on an aligned copy
        const int ldt = (m + 3) & ~3;
        float *ct = nullptr;
        LU_CUDA_TRY(ws.get(&ct, (size_t)ldt * n));
        LU_CUDA_TRY(cudaMemcpy2DAsync(ct, sizeof(float) * ldt, dC, sizeof(float) * ldc, sizeof(float) * m, n,
                                      cudaMemcpyDeviceToDevice, s));
        LU_CUDA_TRY(launch_gemm_tc(nprod, m, n, kpad, ma, 0, mb, 0, ct, ldt, ctr, st->status, lu_spin_bound_ns(nullptr), s,
                                   scA, scB));
        LU_CUDA_TRY(cudaMemcpy2DAsync(dC, sizeof(float) * ldc, ct, sizeof(float) * ldt, sizeof(float) * m, n,
                                      cudaMemcpyDeviceToDevice, s));
    }
    return LU_OK;
}

int lu_trailing_update_f64(int update, int m, int n, int k, const double *dA, int lda, const double *dB, int ldb,
                           double *dC, int ldc, void *stream) {
    if (update != LU_UPDATE_NATIVE && update != LU_UPDATE_F64EMU) return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (k < 0 || (update == LU_UPDATE_F64EMU && k > f64emu_kpad())) return -4;
    if (m > 0 && k > 0 && !dA) return -5;
    if (lda < std::max(1, m)) return -6;
    if (n > 0 && k > 0 && !dB) return -7;
    if (ldb < std::max(1, k)) return -8;
    if (m > 0 && n > 0 && !dC) return -9;
    if (ldc < std::max(1, m)) return -10;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (m == 0 || n == 0 || k == 0) return LU_OK;
    if (update == LU_UPDATE_NATIVE) {
        LU_CUDA_TRY(launch_gemm_simt<double>(m, n, k, dA, lda, dB, ldb, dC, ldc, s));
        return LU_OK;
    }
    DevState *st = nullptr;
    LU_CUDA_TRY(dev_state(&st));
    Workspace ws(s);
    const int kinner = f64emu_kpad() * kF64Slices;
    __nv_bfloat16 *sa = nullptr, *sb = nullptr;
    double *scA = nullptr, *scB = nullptr;
    int *ctr = nullptr;
    LU_CUDA_TRY(ws.get(&sa, (size_t)m * kinner));
    LU_CUDA_TRY(ws.get(&sb, (size_t)n * kinner));
    LU_CUDA_TRY(ws.get(&scA, (size_t)m));
    LU_CUDA_TRY(ws.get(&scB, (size_t)n));
    LU_CUDA_TRY(ws.get(&ctr, 1));
    LU_CUDA_TRY(launch_stage_rows_f64emu(m, k, dA, lda, sa, kinner, scA, s));
    LU_CUDA_TRY(launch_stage_cols_f64emu(k, n, dB, ldb, sb, kinner, scB, s));
    CUtensorMap ma, mb;
    LU_CUDA_TRY(make_stage_map(&ma, sa, kinner, m, kinner, f64emu_box_rows(), 0));
    LU_CUDA_TRY(make_stage_map(&mb, sb, kinner, n, kinner, f64emu_box_cols(), 0));
    LU_CUDA_TRY(launch_gemm_f64emu(m, n, ma, 0, mb, 0, dC, ldc, scA, scB, ctr, st->status, lu_spin_bound_ns(nullptr), 0, s));
    return LU_OK;
}

size_t lu_workspace_size(const char *routine, int n, int nrhs, lu_dtype dt) {
    if (!routine || n < 0 || nrhs < 0) return 0;
    const size_t N = (size_t)n, elem = dt == LU_F64 ? 8 : 4;
    if (!strcmp(routine, "factor")) return 3 * (1 + 4 * 256) * sizeof(int) + (dt == LU_F32 ? 3 * N * 512 * 2 : 0);
    if (!strcmp(routine, "solve")) return N * sizeof(int) + N * nrhs * elem + trsv_workspace_ints(n, nrhs) * sizeof(int);
    if (!strcmp(routine, "mixed"))
        return N * N * 4 + N * sizeof(int) * 2 + 3 * N * 512 * 2 + residual_workspace_doubles(n, nrhs) * 8 +
               N * nrhs * (8 * 2 + 4 * 2) + N * 8;
    return 0;
}

const char *lu_status_string(int code) {
    switch (code) {
        case LU_OK: return "success";
        case LU_ERR_CUDA: return "CUDA runtime error";
        case LU_ERR_NOMEM: return "workspace allocation failed";
        case LU_ERR_TIMEOUT: return "a bounded device-side wait expired";
        case LU_ERR_UNSUPPORTED: return "unsupported request";
        case LU_ERR_SCRATCH: return "request exceeds the fixed scratch of the no-allocation entry point";
        default: break;
    }
    if (code < 0 && code > -100) return "invalid argument (return value -i names argument i)";
    return "unknown status";
}

int lu_wait_selftest(long long bound_ns, void *stream) {
    if (bound_ns <= 0) return -1;
    DevState *st = nullptr;
    LU_CUDA_TRY(dev_state(&st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = 2 * 64;   // two row blocks: block 1 waits on block 0, which nobody solves
    Workspace ws(s);
    float *LU = nullptr, *X = nullptr;
    int *tw = nullptr, *status = nullptr;
    LU_CUDA_TRY(ws.get(&LU, (size_t)n * n));
    LU_CUDA_TRY(ws.get(&X, (size_t)n));
    LU_CUDA_TRY(ws.get(&tw, trsv_workspace_ints(n, 1)));
    LU_CUDA_TRY(ws.get(&status, 1));
    LU_CUDA_TRY(cudaMemsetAsync(LU, 0, sizeof(float) * n * n, s));
    LU_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(float) * n, s));
    LU_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    LU_CUDA_TRY(launch_trsv_timeout_selftest(LU, n, X, tw, status, bound_ns, s));
    int v = 0;
    LU_CUDA_TRY(cudaMemcpyAsync(&v, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaStreamSynchronize(s));
    return v;
}

long long lu_div_selftest(lu_dtype dt, long long count, unsigned long long seed, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (count < 0) return -2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    unsigned long long *bad = nullptr;
    LU_CUDA_TRY(ws.get(&bad, 1));
    LU_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
    LU_CUDA_TRY(launch_div_selftest(dt == LU_F64, count, seed, bad, s));
    unsigned long long h = 0;
    LU_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaStreamSynchronize(s));
    return (long long)h;
}

int lu_last_device_status(void *stream, int reset) {
    DevState *st = nullptr;
    LU_CUDA_TRY(dev_state(&st));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int v = 0;
    LU_CUDA_TRY(cudaMemcpyAsync(&v, st->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    LU_CUDA_TRY(cudaStreamSynchronize(s));
    if (reset) LU_CUDA_TRY(cudaMemsetAsync(st->status, 0, sizeof(int), s));
    return v;
}

int lu_get_status(void *stream) { return lu_last_device_status(stream, 0); }

int lu_update_timing(int enable) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timing = enable != 0;
    return LU_OK;
}

int lu_update_timing_read(long long *launches, double *total_ms, double *flops, double *bytes) {
    std::vector<TimedLaunch> v;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        v.swap(g_timed);
    }
    double ms = 0.0, fl = 0.0, by = 0.0;
    int rc = LU_OK;
    for (auto &t : v) {
        float e = 0.f;
        cudaError_t st = cudaEventSynchronize(t.b);
        if (st == cudaSuccess) st = cudaEventElapsedTime(&e, t.a, t.b);
        if (st != cudaSuccess) rc = LU_ERR_CUDA;
        ms += e;
        fl += t.flops;
        by += t.bytes;
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    if (launches) *launches = (long long)v.size();
    if (total_ms) *total_ms = ms;
    if (flops) *flops = fl;
    if (bytes) *bytes = by;
    return rc;
}

int lu_trace(int enable) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_trace_on = enable != 0;
    return LU_OK;
}

int lu_trace_read(lu_trace_event *out, int max_events) {
    std::vector<TraceRec> v;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        v.swap(g_trace);
    }
    int rc = LU_OK;
    for (auto &t : v)
        if (cudaEventSynchronize(t.b) != cudaSuccess) rc = LU_ERR_CUDA;
    int nout = 0;
    if (rc == LU_OK && !v.empty()) {
        // origin: the earliest start event
        size_t o = 0;
        for (size_t i = 1; i < v.size(); ++i) {
            float d = 0.f;
            if (cudaEventElapsedTime(&d, v[o].a, v[i].a) == cudaSuccess && d < 0.f) o = i;
        }
        for (size_t i = 0; i < v.size() && out && nout < max_events; ++i) {
            float t0 = 0.f, t1 = 0.f;
            if (cudaEventElapsedTime(&t0, v[o].a, v[i].a) != cudaSuccess ||
                cudaEventElapsedTime(&t1, v[o].a, v[i].b) != cudaSuccess) {
                rc = LU_ERR_CUDA;
                break;
            }
            out[nout++] = lu_trace_event{v[i].kind, v[i].step, v[i].stream, t0, t1};
        }
    }
    for (auto &t : v) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    return rc == LU_OK ? (out ? nout : (int)v.size()) : rc;
}

int lu_cta_trace(int capacity) {
    if (capacity < 0) return -1;
    std::lock_guard<std::mutex> lk(g_tmu);
    if (g_cta.ring) {
        int d = -1;
        cudaGetDevice(&d);
        cudaSetDevice(g_cta.dev);
        cudaDeviceSynchronize();
        cudaFree(g_cta.ring);
        cudaFree(g_cta.count);
        cudaSetDevice(d);
        g_cta = CtaRing{};
    }
    if (capacity == 0) return LU_OK;
    CtaRing r;
    LU_CUDA_TRY(cudaGetDevice(&r.dev));
    if (cudaMalloc(&r.ring, sizeof(lu_cta_event) * (size_t)capacity) != cudaSuccess) return LU_ERR_NOMEM;
    if (cudaMalloc(&r.count, sizeof(int)) != cudaSuccess) {
        cudaFree(r.ring);
        return LU_ERR_NOMEM;
    }
    LU_CUDA_TRY(cudaMemset(r.count, 0, sizeof(int)));
    r.cap = capacity;
    g_cta = r;
    return LU_OK;
}

int lu_cta_trace_read(lu_cta_event *out, int max_events) {
    std::lock_guard<std::mutex> lk(g_tmu);
    if (!g_cta.ring) return 0;
    int d = -1;
    LU_CUDA_TRY(cudaGetDevice(&d));
    LU_CUDA_TRY(cudaSetDevice(g_cta.dev));
    LU_CUDA_TRY(cudaDeviceSynchronize());
    int made = 0;
    LU_CUDA_TRY(cudaMemcpy(&made, g_cta.count, sizeof(int), cudaMemcpyDeviceToHost));
    const int avail = std::min(made, g_cta.cap);
    if (out && max_events > 0 && avail > 0)
        LU_CUDA_TRY(cudaMemcpy(out, g_cta.ring, sizeof(lu_cta_event) * (size_t)std::min(avail, max_events),
                               cudaMemcpyDeviceToHost));
    LU_CUDA_TRY(cudaMemset(g_cta.count, 0, sizeof(int)));
    LU_CUDA_TRY(cudaSetDevice(d));
    return made;
}

long long lu_kernel_launches(void) { return g_launches.load(); }

const char *lu_version(void) {
    return "liblu 0.2 (sm_103a; cluster panel, tcgen05 BF16 / split-BF16 / FP8 and emulated FP64 updates, FP64 DFMA update)";
}

size_t lu_abi_size(const char *name) {
    if (!name) return 0;
    if (!strcmp(name, "lu_opts")) return sizeof(lu_opts);
    if (!strcmp(name, "lu_mixed_opts")) return sizeof(lu_mixed_opts);
    if (!strcmp(name, "lu_mixed_report")) return sizeof(lu_mixed_report);
    if (!strcmp(name, "lu_tune_result")) return sizeof(lu_tune_result);
    if (!strcmp(name, "lu_trace_event")) return sizeof(lu_trace_event);
    if (!strcmp(name, "lu_cta_event")) return sizeof(lu_cta_event);
    return 0;
}

}  // extern "C"

// internal entry points used by the mixed-precision driver (mixed_api.cu) and
// the Cholesky factorization (cholesky.cu)
namespace lu {
CtaTrace cta_tag_ext(int kind, int step) { return cta_tag(kind, step); }
int factor_f32_internal(int n, float *A, int lda, int *ipiv, int *info, int *perm, const lu_opts *o, cudaStream_t s) {
    lu_opts tuned;
    o = with_tuned(0, LU_F32, n, o, &tuned);
    Plan p = make_plan<float>(n, o);
    return factor_impl<float>(n, A, lda, ipiv, info, perm, p, s);
}
int factor_f64_internal(int n, double *A, int lda, int *ipiv, int *info, int *perm, const lu_opts *o, cudaStream_t s) {
    lu_opts tuned;
    o = with_tuned(0, LU_F64, n, o, &tuned);
    Plan p = make_plan<double>(n, o);
    return factor_impl<double>(n, A, lda, ipiv, info, perm, p, s);
}
int default_outer_width(lu_dtype dt, int n, int update) {
    lu_opts o = {};
    o.update = update;
    return dt == LU_F64 ? make_plan<double>(n, &o).bo : make_plan<float>(n, &o).bo;
}
int solve_f32_perm(int n, int nrhs, const float *LU, int lda, const int *perm, float *B, int ldb, cudaStream_t s,
                   const float *Dinv) {
    return solve_impl<float>(n, nrhs, LU, lda, nullptr, perm, B, ldb, lu_spin_bound_ns(nullptr), s, Dinv);
}
// Dinv := the inverses of the FP32 factors' 64 x 64 diagonal blocks (for solve_f32_perm)
size_t f32_diag_inverse_elems(int n) { return trsv_inverse_elems<float>(n); }
int f32_diag_inverse(int n, const float *LU, int lda, float *Dinv, cudaStream_t s) {
    LU_CUDA_TRY(launch_diag_inverse<float>(LU, lda, n, Dinv, s));
    return LU_OK;
}
int solve_f64_perm(int n, int nrhs, const double *LU, int lda, const int *perm, double *B, int ldb, cudaStream_t s,
                   const double *Dinv) {
    return solve_impl<double>(n, nrhs, LU, lda, nullptr, perm, B, ldb, lu_spin_bound_ns(nullptr), s, Dinv);
}
size_t f64_diag_inverse_elems(int n) { return trsv_inverse_elems<double>(n); }
int f64_diag_inverse(int n, const double *LU, int lda, double *Dinv, cudaStream_t s) {
    LU_CUDA_TRY(launch_diag_inverse<double>(LU, lda, n, Dinv, s));
    return LU_OK;
}
}  // namespace lu
