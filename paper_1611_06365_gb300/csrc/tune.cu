// Autotuner: the block-size tension of section 3.1 (a wide panel b_o makes a
// fast update, a narrow one makes a short panel chain) and the size of the
// panel team of section 3.2 are settled by measurement on the device at hand.
// lu_autotune times lu_factor on a scratch matrix of the requested order for a
// small set of candidate plans; the fastest goes into a process-wide table that
// lu_factor and lu_factor_batched consult for every option left at zero.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "lu.h"

#include "internal.h"

namespace {

using Key = std::tuple<int, int, int, int>;   // kind, dtype, update, n
struct Entry {
    lu_opts o;
    double ms;
};
std::mutex g_tmu;
std::map<Key, Entry> g_table;
thread_local bool g_bypass = false;   // set while the tuner times its candidates

// Scratch entries uniform in [-1, 1): splitmix64 (Steele, Lea and Flood,
// OOPSLA 2014) of the element index; the values only need to look like the
// workload to the pivot search.
template <typename T>
__global__ void tune_fill(T *A, size_t count, unsigned long long seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        A[i] = T(2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0);
    }
}

template <typename T>
cudaError_t fill(void *A, size_t count, unsigned long long seed, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int blocks = (int)std::min<size_t>((count + 255) / 256, 4096);
    tune_fill<T><<<blocks, 256, 0, s>>>(static_cast<T *>(A), count, seed);
    lu_count_launch(1);
    return cudaGetLastError();
}

bool valid_update(lu_dtype dt, int update) {
    if (update == LU_UPDATE_NATIVE) return true;
    if (update == LU_UPDATE_F64EMU) return dt == LU_F64;
    return dt == LU_F32 && (update == LU_UPDATE_BF16 || update == LU_UPDATE_BF16X3 || update == LU_UPDATE_FP8);
}

lu_opts make_opts(int nb, int nb_inner, int panel_ctas, int lookahead, int update, int update_ctas = 0, int tile = 0) {
    lu_opts o = {};
    o.tile = tile;
    o.nb = nb;
    o.nb_inner = nb_inner;
    o.panel_ctas = panel_ctas;
    o.lookahead = lookahead;
    o.update = update;
    o.update_ctas = update_ctas;
    return o;
}

bool opts_in_range(int kind, const lu_opts &o) {
    if (o.nb < 0 || o.nb_inner < 0 || o.panel_ctas < 0 || o.panel_ctas > 16 || o.lookahead < -1 || o.lookahead > 4 ||
        o.update_ctas < 0 || o.update_ctas > 4096 || o.tile < 0 || o.tile > 2)
        return false;
    return kind != 1 || o.nb == 0 || o.nb == 1 || o.nb == 16 || o.nb == 32;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" {

int lu_tune_get(int kind, lu_dtype dt, int update, int n, lu_opts *out) {
    if (g_bypass || !out) return 0;
    std::lock_guard<std::mutex> lk(g_tmu);
    auto it = g_table.find(Key{kind, (int)dt, update, n});
    if (it == g_table.end()) return 0;
    *out = it->second.o;
    return 1;
}

int lu_tune_put(int kind, lu_dtype dt, int update, int n, const lu_opts *o, double ms) {
    if (kind != 0 && kind != 1) return -1;
    if (dt != LU_F64 && dt != LU_F32) return -2;
    if (!valid_update(dt, update)) return -3;
    if (n < 0) return -4;
    if (!o || !opts_in_range(kind, *o)) return -5;
    lu_opts c = make_opts(o->nb, o->nb_inner, o->panel_ctas, o->lookahead, update, o->update_ctas, o->tile);
    std::lock_guard<std::mutex> lk(g_tmu);
    g_table[Key{kind, (int)dt, update, n}] = Entry{c, ms};
    return LU_OK;
}

void lu_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_table.clear();
}

int lu_tune_count(void) {
    std::lock_guard<std::mutex> lk(g_tmu);
    return (int)g_table.size();
}

int lu_tune_save(const char *path) {
    if (!path) return -1;
    FILE *f = fopen(path, "w");
    if (!f) return -1;
    std::lock_guard<std::mutex> lk(g_tmu);
    fprintf(f, "# liblu tuning table v2\n# kind dtype update n nb nb_inner panel_ctas lookahead update_ctas tile ms\n");
    for (const auto &kv : g_table) {
        const lu_opts &o = kv.second.o;
        fprintf(f, "%d %d %d %d %d %d %d %d %d %d %.6f\n", std::get<0>(kv.first), std::get<1>(kv.first),
                std::get<2>(kv.first), std::get<3>(kv.first), o.nb, o.nb_inner, o.panel_ctas, o.lookahead, o.update_ctas,
                o.tile, kv.second.ms);
    }
    const int bad = ferror(f);
    fclose(f);
    return bad ? -1 : (int)g_table.size();
}

int lu_tune_load(const char *path) {
    if (!path) return -1;
    FILE *f = fopen(path, "r");
    if (!f) return -1;
    struct Row {
        int kind, dt, update, n;
        lu_opts o;
        double ms;
    };
    std::vector<Row> rows;
    char line[512];
    bool ok = true;
    while (fgets(line, sizeof(line), f)) {
        const char *p = line;
        while (*p == ' ' || *p == '\t') ++p;
        if (*p == '#' || *p == '\n' || *p == '\r' || *p == '\0') continue;
        Row r{};
        char tail = 0;
        // v2 lines carry the tile shape before ms (11 fields); v1 lines have 10 and mean tile 0
        int fields = 0;
        for (const char *q = p; *q;) {
            while (*q == ' ' || *q == '\t' || *q == '\n' || *q == '\r') ++q;
            if (!*q) break;
            ++fields;
            while (*q && *q != ' ' && *q != '\t' && *q != '\n' && *q != '\r') ++q;
        }
        int got = -1;
        if (fields == 11)
            got = sscanf(p, "%d %d %d %d %d %d %d %d %d %d %lf %c", &r.kind, &r.dt, &r.update, &r.n, &r.o.nb,
                         &r.o.nb_inner, &r.o.panel_ctas, &r.o.lookahead, &r.o.update_ctas, &r.o.tile, &r.ms, &tail);
        else if (fields == 10)
            got = 1 + sscanf(p, "%d %d %d %d %d %d %d %d %d %lf %c", &r.kind, &r.dt, &r.update, &r.n, &r.o.nb,
                             &r.o.nb_inner, &r.o.panel_ctas, &r.o.lookahead, &r.o.update_ctas, &r.ms, &tail);
        if (got != 11) {
            ok = false;
            break;
        }
        rows.push_back(r);
    }
    fclose(f);
    if (!ok) return -2;
    // validate every row before taking any (a file is taken whole or not at all)
    for (const Row &r : rows) {
        const lu_dtype dt = (lu_dtype)r.dt;
        if ((r.kind != 0 && r.kind != 1) || (r.dt != LU_F64 && r.dt != LU_F32) || !valid_update(dt, r.update) || r.n < 0 ||
            !opts_in_range(r.kind, r.o))
            return -2;
    }
    for (const Row &r : rows) lu_tune_put(r.kind, (lu_dtype)r.dt, r.update, r.n, &r.o, r.ms);
    return (int)rows.size();
}

int lu_autotune(lu_dtype dt, int n, int update, double budget_ms, lu_tune_result *res, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (n < 1) return -2;
    if (!valid_update(dt, update)) return -3;
    if (!res) return -5;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t elem = dt == LU_F64 ? 8 : 4;
    const size_t count = (size_t)n * n;

    // candidates: the built-in plan first, then the other outer widths, then
    // smaller panel teams around the best width
    std::vector<int> widths;
    if (update == LU_UPDATE_F64EMU) widths = {32, 64};   // the emulated update takes K <= 64
    else if (update != LU_UPDATE_NATIVE) widths = {64, 128, 256};
    else if (dt == LU_F32) widths = {64, 128, 256};
    else widths = {16, 32, 64};
    const int nb0 = lu::default_outer_width(dt, n, update);
    std::vector<lu_opts> cands;
    cands.push_back(make_opts(0, 0, 0, 0, update));
    for (int w : widths)
        if (w != nb0 && w <= n) cands.push_back(make_opts(w, 0, 0, 0, update));

    void *A0 = nullptr, *A = nullptr;
    int *ipiv = nullptr, *info = nullptr;
    int rc = LU_OK;
    Timer t;
    double best_ms = 1e300;
    lu_opts best = cands[0];
    int timed = 0;
    double spent = 0.0;
    const bool small = n <= 4096;   // short runs: one warm-up and the best of three
    auto run = [&](const lu_opts &o, double *ms) -> int {
        float best_rep = 1e30f;
        const int reps = small ? 3 : 1;
        for (int r = (small ? -1 : 0); r < reps; ++r) {
            if (cudaMemcpyAsync(A, A0, count * elem, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return LU_ERR_CUDA;
            if (cudaEventRecord(t.a, s) != cudaSuccess) return LU_ERR_CUDA;
            const int e = lu_factor(dt, n, A, n, ipiv, info, &o, s);
            if (e != LU_OK) return e;
            if (cudaEventRecord(t.b, s) != cudaSuccess) return LU_ERR_CUDA;
            if (cudaEventSynchronize(t.b) != cudaSuccess) return LU_ERR_CUDA;
            float m = 0.f;
            if (cudaEventElapsedTime(&m, t.a, t.b) != cudaSuccess) return LU_ERR_CUDA;
            spent += m;
            if (r >= 0) best_rep = std::min(best_rep, m);
        }
        *ms = best_rep;
        return LU_OK;
    };
    auto consider = [&](const lu_opts &o) -> int {
        if (timed > 0 && budget_ms > 0 && spent >= budget_ms) return LU_OK;
        double ms = 0;
        const int e = run(o, &ms);
        if (e == LU_ERR_CUDA || e == LU_ERR_TIMEOUT) return e;
        if (e != LU_OK) return LU_OK;   // a plan this order cannot take: skip it
        ++timed;
        if (ms < best_ms) {
            best_ms = ms;
            best = o;
        }
        return LU_OK;
    };

    g_bypass = true;
    do {
        if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) { rc = LU_ERR_CUDA; break; }
        if (cudaMallocAsync(&A0, count * elem, s) != cudaSuccess || cudaMallocAsync(&A, count * elem, s) != cudaSuccess ||
            cudaMallocAsync(&ipiv, sizeof(int) * n, s) != cudaSuccess || cudaMallocAsync(&info, sizeof(int), s) != cudaSuccess) {
            rc = LU_ERR_NOMEM;
            break;
        }
        if ((dt == LU_F64 ? fill<double>(A0, count, 20161106ull + (unsigned)n, s)
                          : fill<float>(A0, count, 20161106ull + (unsigned)n, s)) != cudaSuccess) {
            rc = LU_ERR_CUDA;
            break;
        }
        for (const lu_opts &o : cands)
            if ((rc = consider(o)) != LU_OK) break;
        if (rc != LU_OK) break;
        for (int pc : {8, 4})
            if ((rc = consider(make_opts(best.nb, 0, pc, best.lookahead, update))) != LU_OK) break;
        if (rc != LU_OK) break;
        if (n <= 2048 && (rc = consider(make_opts(best.nb, 0, best.panel_ctas, -1, update))) != LU_OK) break;
        // depth-2 look-ahead (section 3.2's look-ahead over more than one panel)
        if (best.lookahead >= 0 && (rc = consider(make_opts(best.nb, 0, best.panel_ctas, 2, update))) != LU_OK) break;
        // tensor-core updates: leave some SMs to the panel chain (a smaller RU2 grid)
        if (update != LU_UPDATE_NATIVE &&
            (rc = consider(make_opts(best.nb, 0, best.panel_ctas, best.lookahead, update, 112))) != LU_OK)
            break;
        // the update's tile shape (DFMA tiles, emulated FP64 task length)
        if (update == LU_UPDATE_NATIVE || update == LU_UPDATE_F64EMU)
            for (int tl : {1, 2})
                if ((rc = consider(make_opts(best.nb, 0, best.panel_ctas, best.lookahead, update, best.update_ctas, tl))) !=
                    LU_OK)
                    break;
        if (rc != LU_OK) break;
    } while (false);
    g_bypass = false;
    if (A0) cudaFreeAsync(A0, s);
    if (A) cudaFreeAsync(A, s);
    if (ipiv) cudaFreeAsync(ipiv, s);
    if (info) cudaFreeAsync(info, s);
    if (rc != LU_OK) return rc;
    if (timed == 0) return LU_ERR_UNSUPPORTED;
    if (best.nb == 0) best.nb = nb0;
    lu_tune_put(0, dt, update, n, &best, best_ms);
    res->opts = best;
    res->ms = best_ms;
    res->candidates = timed;
    return LU_OK;
}

int lu_autotune_batched(lu_dtype dt, int batch, const int *d_n, int max_n, lu_tune_result *res, void *stream) {
    if (dt != LU_F64 && dt != LU_F32) return -1;
    if (batch < 1) return -2;
    if (!d_n) return -3;
    if (max_n < 1 || max_n > 1024) return -4;
    if (!res) return -5;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t elem = dt == LU_F64 ? 8 : 4;
    std::vector<int> ns(batch);
    if (cudaMemcpyAsync(ns.data(), d_n, sizeof(int) * batch, cudaMemcpyDeviceToHost, s) != cudaSuccess) return LU_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LU_ERR_CUDA;
    std::vector<size_t> off(batch + 1, 0), poff(batch + 1, 0);
    std::vector<int> ld(batch);
    for (int t = 0; t < batch; ++t) {
        if (ns[t] < 0 || ns[t] > max_n) return -3;
        ld[t] = std::max(1, ns[t]);
        off[t + 1] = off[t] + (size_t)ld[t] * ld[t];
        poff[t + 1] = poff[t] + (size_t)ld[t];
    }
    std::vector<int> nbs;
    if (max_n <= 256) nbs = {16, 32, 1};
    else nbs = {1};

    unsigned char *A0 = nullptr, *A = nullptr;
    int *ipiv = nullptr, *info = nullptr, *dld = nullptr;
    unsigned long long *pA = nullptr, *pP = nullptr;
    int rc = LU_OK;
    Timer t;
    double best_ms = 1e300;
    int best_nb = nbs[0], timed = 0;
    g_bypass = true;
    do {
        if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) { rc = LU_ERR_CUDA; break; }
        if (cudaMallocAsync(&A0, off[batch] * elem, s) != cudaSuccess || cudaMallocAsync(&A, off[batch] * elem, s) != cudaSuccess ||
            cudaMallocAsync(&ipiv, sizeof(int) * poff[batch], s) != cudaSuccess ||
            cudaMallocAsync(&info, sizeof(int) * batch, s) != cudaSuccess || cudaMallocAsync(&dld, sizeof(int) * batch, s) != cudaSuccess ||
            cudaMallocAsync(&pA, sizeof(unsigned long long) * batch, s) != cudaSuccess ||
            cudaMallocAsync(&pP, sizeof(unsigned long long) * batch, s) != cudaSuccess) {
            rc = LU_ERR_NOMEM;
            break;
        }
        std::vector<unsigned long long> ha(batch), hp(batch);
        for (int tt = 0; tt < batch; ++tt) {
            ha[tt] = (unsigned long long)(A + off[tt] * elem);
            hp[tt] = (unsigned long long)(ipiv + poff[tt]);
        }
        if (cudaMemcpyAsync(pA, ha.data(), sizeof(unsigned long long) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(pP, hp.data(), sizeof(unsigned long long) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(dld, ld.data(), sizeof(int) * batch, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            rc = LU_ERR_CUDA;
            break;
        }
        if ((dt == LU_F64 ? fill<double>(A0, off[batch], 20161106ull, s) : fill<float>(A0, off[batch], 20161106ull, s)) !=
            cudaSuccess) {
            rc = LU_ERR_CUDA;
            break;
        }
        for (int nb : nbs) {
            lu_opts o = make_opts(nb, 0, 0, 0, 0);
            float best_rep = 1e30f;
            for (int r = -1; r < 3 && rc == LU_OK; ++r) {
                if (cudaMemcpyAsync(A, A0, off[batch] * elem, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                    cudaEventRecord(t.a, s) != cudaSuccess) {
                    rc = LU_ERR_CUDA;
                    break;
                }
                const int e = lu_factor_batched(dt, batch, d_n, reinterpret_cast<void *const *>(pA), dld,
                                                reinterpret_cast<int *const *>(pP), info, max_n, &o, s);
                if (e != LU_OK) { rc = e; break; }
                float m = 0.f;
                if (cudaEventRecord(t.b, s) != cudaSuccess || cudaEventSynchronize(t.b) != cudaSuccess ||
                    cudaEventElapsedTime(&m, t.a, t.b) != cudaSuccess) {
                    rc = LU_ERR_CUDA;
                    break;
                }
                if (r >= 0) best_rep = std::min(best_rep, m);
            }
            if (rc != LU_OK) break;
            ++timed;
            if (best_rep < best_ms) {
                best_ms = best_rep;
                best_nb = nb;
            }
        }
    } while (false);
    g_bypass = false;
    for (void *p : {(void *)A0, (void *)A, (void *)ipiv, (void *)info, (void *)dld, (void *)pA, (void *)pP})
        if (p) cudaFreeAsync(p, s);
    if (rc != LU_OK) return rc;
    lu_opts best = make_opts(best_nb, 0, 0, 0, 0);
    lu_tune_put(1, dt, 0, max_n, &best, best_ms);
    res->opts = best;
    res->ms = best_ms;
    res->candidates = timed;
    return LU_OK;
}

}  // extern "C"
