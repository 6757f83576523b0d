// C-ABI implementation (include/pastila.h): handles, device memory, launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/pastila.h"
#include <nvtx3/nvToolsExt.h>  // header-only: ranges cost a branch unless a profiler is attached
#include "batch.cuh"
#include "keys.cuh"
#include "probe.cuh"
#include "snippets.cuh"
#include "stats.cuh"
#include "tile.cuh"

using namespace pastila;

namespace {

// A named NVTX range over a scope (host side: marks when each phase is enqueued;
// profilers show it beside the kernels it launched).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

thread_local std::string g_err;

pastila_status fail(pastila_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(PASTILA_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                            \
    } while (0)

#define TRY(...)                                \
    do {                                        \
        pastila_status st_ = (__VA_ARGS__);     \
        if (st_ != PASTILA_OK) return st_;      \
    } while (0)

constexpr int V_F32 = 4;
constexpr int V_F64 = 4;
constexpr int MAX_NT = 512;
constexpr int64_t ARRAY_PAD = 16;  // elements past the end of every array a tile stages

// The bounded waits of the tile kernels: about a second of SM cycles, or, with
// PASTILA_TEST_STAGE_WAIT=timeout in the environment when a handle or an
// engine is created, an added wait on a phase that nothing completes, with a
// limit of about half a millisecond (the test that makes the wait run out).
void wait_knobs(long long* spin_limit, int* test_timeout) {
    const char* t = getenv("PASTILA_TEST_STAGE_WAIT");
    const bool test = t && !strcmp(t, "timeout");
    *test_timeout = test ? 1 : 0;
    *spin_limit = test ? (1ll << 20) : (1ll << 31);
}

// Launch of a tile kernel: plain for one-CTA tiles, with clusters of cs CTAs
// (along x) otherwise.
template <typename... P, typename... Q>
cudaError_t launch_tiles(void (*kernel)(P...), dim3 grid, unsigned block, size_t smem, cudaStream_t st, int cs,
                         Q&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs > 1 ? cs : 1;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = cs > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Q>(args)...);
}

// Shared-memory attributes of a tile kernel: up to `smem` dynamic bytes per CTA,
// and the largest shared-memory carveout, so that two CTAs of a layout that
// needs at most half of it share an SM.
template <typename... P>
cudaError_t tile_attrs(void (*kernel)(P...), int smem) {
    cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (r != cudaSuccess) return r;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

struct Stats {
    bool stale = false;
    int64_t C = 0;
    double* mu = nullptr;
    void* a = nullptr;
    void* df = nullptr;
    void* dg = nullptr;
    void* muh = nullptr;  // mu as hi + lo pairs of the handle's precision
    void* mul = nullptr;
};

struct Buf {
    void* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct pastila_series {
    int device = 0;
    pastila_precision prec = PASTILA_FP32;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t n = 0;
    double* T = nullptr;
    void* Th = nullptr;  // T as hi + lo pairs of the handle's precision, rewritten with every statistic
    void* Tl = nullptr;
    int* err = nullptr;  // host-mapped flag the tile kernels set when a bounded wait runs out
    long long spin_limit = 1ll << 31;  // SM cycles (about a second)
    int test_timeout = 0;
    size_t budget = 0;
    size_t held = 0;
    int smem_optin = 0;
    uint64_t launches = 0;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<cudaEvent_t> ev_free;
    double tile_ms = 0.0;
    int64_t tile_launches = 0;
    double tile_cells = 0.0;
    std::map<int, Stats> stats;
    // FP64 statistics of an FP32 handle (the FP64 re-evaluation of near-tied
    // greedy steps), with T as FP64 pairs (value, 0)
    std::map<int, Stats> stats64;
    void* Th64 = nullptr;
    void* Tl64 = nullptr;
    int phase2_launches = 0;  // kernels of the last enqueued greedy phase of a sweep
    bool fp64_ties = true;    // FP32 handles: near-tied greedy steps decided on FP64 areas
    std::map<std::string, Buf> bufs;
    uint64_t alloc_gen = 0;  // bumped whenever a device buffer is (re)allocated
    // captured select_length sequence, replayed while the configuration and the
    // buffers it references stay the same
    struct {
        std::vector<int32_t> ms;
        pastila_mparams rule{0, 0};
        int K = 0;
        uint64_t gen = ~0ull;
        uint64_t tune_gen = ~0ull;  // the autotuner's table when the graphs were made
        cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};  // statistics, tiles, snippets
        int calls = 0;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the tile graph, while timing is on
    } graph;
};

namespace {

size_t real_size(const pastila_series* h) { return h->prec == PASTILA_FP64 ? 8 : 4; }

pastila_status dev_alloc(pastila_series* h, void** p, size_t bytes) {
    if (h->budget && h->held + bytes > h->budget)
        return fail(PASTILA_ENOMEM, "memory budget exceeded: need %zu more bytes, hold %zu of %zu",
                    bytes, h->held, h->budget);
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(PASTILA_ENOMEM, "cudaMalloc(%zu) failed: out of device memory", bytes);
    }
    if (e != cudaSuccess) return fail(PASTILA_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    h->held += bytes;
    h->alloc_gen++;
    return PASTILA_OK;
}

void dev_free(pastila_series* h, void* p, size_t bytes) {
    if (p) {
        cudaFree(p);
        h->held -= bytes;
    }
}

// Named scratch buffer that only grows.
pastila_status scratch(pastila_series* h, const char* name, size_t bytes, void** out) {
    Buf& b = h->bufs[name];
    if (b.n < bytes) {
        CK(cudaStreamSynchronize(h->stream));
        dev_free(h, b.p, b.n);
        b.p = nullptr;
        b.n = 0;
        TRY(dev_alloc(h, &b.p, bytes));
        b.n = bytes;
    }
    *out = b.p;
    return PASTILA_OK;
}

pastila_status set_device(const pastila_series* h) {
    CK(cudaSetDevice(h->device));
    return PASTILA_OK;
}

// After the handle's stream is synchronised: a tile whose bounded wait ran out
// leaves results that must not be used.
pastila_status stage_check(pastila_series* h) {
    if (!*(volatile int*)h->err) return PASTILA_OK;
    *(volatile int*)h->err = 0;
    return fail(PASTILA_ETIMEOUT, "a tile's staging copies did not complete within the wait limit; the outputs are "
                "unspecified");
}

void invalidate_stats(pastila_series* h) {
    for (auto& kv : h->stats) kv.second.stale = true;
    for (auto& kv : h->stats64) kv.second.stale = true;
}

pastila_status ensure_stats(pastila_series* h, int ell, Stats** out) {
    auto it = h->stats.find(ell);
    if (it != h->stats.end() && !it->second.stale) {
        *out = &it->second;
        return PASTILA_OK;
    }
    Stats st;
    st.C = h->n - ell + 1;
    const size_t rs = real_size(h);
    void *mu, *inv, *flat, *a, *df, *dg, *muh, *mul;
    if (it != h->stats.end()) {  // stale: recompute into the same buffers
        mu = it->second.mu;
        a = it->second.a;
        df = it->second.df;
        dg = it->second.dg;
        muh = it->second.muh;
        mul = it->second.mul;
    } else {
        // the tile kernels' bulk copies may read up to 16 bytes past an array's end
        TRY(dev_alloc(h, &mu, 8 * st.C));
        TRY(dev_alloc(h, &a, rs * (st.C + ARRAY_PAD)));
        TRY(dev_alloc(h, &df, rs * (st.C + ARRAY_PAD)));
        TRY(dev_alloc(h, &dg, rs * (st.C + ARRAY_PAD)));
        TRY(dev_alloc(h, &muh, rs * (st.C + ARRAY_PAD)));
        TRY(dev_alloc(h, &mul, rs * (st.C + ARRAY_PAD)));
    }
    if (!h->Th) {
        TRY(dev_alloc(h, &h->Th, rs * (h->n + ARRAY_PAD)));
        TRY(dev_alloc(h, &h->Tl, rs * (h->n + ARRAY_PAD)));
    }
    TRY(scratch(h, "stats_inv", 8 * st.C, &inv));
    TRY(scratch(h, "stats_flat", 4 * st.C, &flat));
    const int64_t nthr = (st.C + STATS_RUN - 1) / STATS_RUN;
    stats_mu_a_kernel<<<(unsigned)((nthr + 127) / 128), 128, 0, h->stream>>>(
        h->T, st.C, ell, (double*)mu, (double*)inv, (int32_t*)flat);
    CK(cudaGetLastError());
    const unsigned nb = (unsigned)((h->n + 255) / 256);
    if (h->prec == PASTILA_FP64)
        stats_terms_kernel<double><<<nb, 256, 0, h->stream>>>(h->T, h->n, st.C, ell, (double*)mu, (double*)inv,
                                                              (double*)a, (double*)df, (double*)dg, (double*)muh,
                                                              (double*)mul, (double*)h->Th, (double*)h->Tl);
    else
        stats_terms_kernel<float><<<nb, 256, 0, h->stream>>>(h->T, h->n, st.C, ell, (double*)mu, (double*)inv,
                                                             (float*)a, (float*)df, (float*)dg, (float*)muh,
                                                             (float*)mul, (float*)h->Th, (float*)h->Tl);
    CK(cudaGetLastError());
    h->launches += 2;
    st.mu = (double*)mu;
    st.a = a;
    st.df = df;
    st.dg = dg;
    st.muh = muh;
    st.mul = mul;
    h->stats[ell] = st;
    *out = &h->stats[ell];
    return PASTILA_OK;
}

// FP64 window statistics of an FP32 handle, for the FP64 rows of the greedy
// re-evaluation (the same kernels as an FP64 handle's statistics).
pastila_status ensure_stats64(pastila_series* h, int ell, Stats** out) {
    auto it = h->stats64.find(ell);
    if (it != h->stats64.end() && !it->second.stale) {
        *out = &it->second;
        return PASTILA_OK;
    }
    Stats st;
    st.C = h->n - ell + 1;
    void *mu, *inv, *flat, *a, *df, *dg, *muh, *mul;
    if (it != h->stats64.end()) {
        mu = it->second.mu;
        a = it->second.a;
        df = it->second.df;
        dg = it->second.dg;
        muh = it->second.muh;
        mul = it->second.mul;
    } else {
        TRY(dev_alloc(h, &mu, 8 * st.C));
        TRY(dev_alloc(h, &a, 8 * (st.C + ARRAY_PAD)));
        TRY(dev_alloc(h, &df, 8 * (st.C + ARRAY_PAD)));
        TRY(dev_alloc(h, &dg, 8 * (st.C + ARRAY_PAD)));
        TRY(dev_alloc(h, &muh, 8 * (st.C + ARRAY_PAD)));
        TRY(dev_alloc(h, &mul, 8 * (st.C + ARRAY_PAD)));
    }
    if (!h->Th64) {
        TRY(dev_alloc(h, &h->Th64, 8 * (h->n + ARRAY_PAD)));
        TRY(dev_alloc(h, &h->Tl64, 8 * (h->n + ARRAY_PAD)));
    }
    TRY(scratch(h, "stats_inv", 8 * st.C, &inv));
    TRY(scratch(h, "stats_flat", 4 * st.C, &flat));
    const int64_t nthr = (st.C + STATS_RUN - 1) / STATS_RUN;
    stats_mu_a_kernel<<<(unsigned)((nthr + 127) / 128), 128, 0, h->stream>>>(
        h->T, st.C, ell, (double*)mu, (double*)inv, (int32_t*)flat);
    stats_terms_kernel<double><<<(unsigned)((h->n + 255) / 256), 256, 0, h->stream>>>(
        h->T, h->n, st.C, ell, (double*)mu, (double*)inv, (double*)a, (double*)df, (double*)dg, (double*)muh,
        (double*)mul, (double*)h->Th64, (double*)h->Tl64);
    CK(cudaGetLastError());
    h->launches += 2;
    st.mu = (double*)mu;
    st.a = a;
    st.df = df;
    st.dg = dg;
    st.muh = muh;
    st.mul = mul;
    h->stats64[ell] = st;
    *out = &h->stats64[ell];
    return PASTILA_OK;
}

struct MParams {
    int m, ell, k, R, S;
    int64_t P, C;
};

// Conditioning ratios of the windows for the FP32 tiles of q (kappa_kernel),
// recomputed from the statistics st on every call (a small launch); nullptr
// for FP64 handles, whose tiles need no check.
pastila_status ensure_kappa(pastila_series* h, const MParams& q, const Stats* st, const float** out) {
    *out = nullptr;
    if (h->prec == PASTILA_FP64) return PASTILA_OK;
    char name[48];
    snprintf(name, sizeof(name), "kappa_%d_%d", q.ell, q.R);
    void* k;
    TRY(scratch(h, name, 4 * (size_t)(q.C + ARRAY_PAD), &k));
    kappa_kernel<float><<<(unsigned)((q.C + 255) / 256), 256, 0, h->stream>>>((const float*)st->a, q.C, q.R,
                                                                            (float*)k);
    CK(cudaGetLastError());
    h->launches += 1;
    *out = (const float*)k;
    return PASTILA_OK;
}

pastila_status resolve_n(int64_t n, int32_t m, pastila_mparams mp, MParams* o) {
    if (m < 4) return fail(PASTILA_EINVAL, "m = %d: must be at least 4", m);
    if ((int64_t)m > n) return fail(PASTILA_EINVAL, "m = %d exceeds the series length %lld", m, (long long)n);
    const int ell = mp.ell ? mp.ell : m / 2;
    const int k = mp.k ? mp.k : (m + 9) / 10;
    if (ell < 2 || ell > m) return fail(PASTILA_EINVAL, "ell = %d: must satisfy 2 <= ell <= m = %d", ell, m);
    if (k < 1) return fail(PASTILA_EINVAL, "k = %d: must be at least 1", k);
    o->m = m;
    o->ell = ell;
    o->k = k;
    o->R = m - ell + 1;
    o->S = (int)(n / m);
    o->P = n - m + 1;
    o->C = n - ell + 1;
    return PASTILA_OK;
}

pastila_status resolve(const pastila_series* h, int32_t m, pastila_mparams mp, MParams* o) {
    return resolve_n(h->n, m, mp, o);
}

// Tile width W and row groups NG: the smallest modelled cost per ED cell of the
// eq. 9 matrix among the layouts that fit the shared memory and 512 threads.
// Rows and seeds are paid on the NTc V columns of a tile (Wb = W + R - 1 rounded
// up to whole warps of column threads; the R - 1 halo columns are recomputed by
// the next tile), the selection on its W
// positions; NG row groups add NG seed rows of ell products per column, and
// fewer than 12 resident warps leave latency exposed.
// Two CTAs of a layout share an SM when each takes at most half of its shared
// memory (the SM has the per-CTA limit plus the 1 KB reserved per CTA; 2 KB
// more are kept for static shared memory) and at most 256 threads (the
// kernels compile to at most 128 registers).  Such layouts are launched apart
// from the others: a launch takes the largest block and shared memory of its
// items.
inline bool pair_layout(const TileGeom& g, size_t limit) {
    return g.NT <= 256 && g.bytes <= (limit + 2048) / 2 - 3072;
}

struct TileCand {
    double cost;  // modelled cost per ED cell
    int W, ngw;   // tile width and the row groups asked of tile_geom
    TileGeom g;
    bool pair;    // two CTAs of this layout fit on one SM
};

constexpr double TUNE_MARGIN = 0.01;
constexpr int CLUSTER_MIN_R = 65;    // two-CTA cluster tiles are considered from R = 65 up
constexpr int CLUSTER4_MIN_R = 129;  // four-CTA cluster tiles from R = 129 up

template <typename real, int V>
void tile_candidates(size_t limit, const MParams& q, std::vector<TileCand>* out, bool clusters = true) {
    out->clear();
    const int64_t Pmax = ((q.P + 31) / 32) * 32;
    for (int cs = 1; cs <= (clusters ? (q.R >= CLUSTER4_MIN_R ? 4 : (q.R >= CLUSTER_MIN_R ? 2 : 1)) : 1); cs *= 2) {
        for (int W = 32; W <= MAX_NT * V && W <= Pmax; W += 32) {
            const int Wb = W + q.R - 1;
            const int NTc = ((Wb + V - 1) / V + 31) / 32 * 32;
            if (NTc > MAX_NT) break;
            const int ng_max = MAX_NT / NTc;
            for (int ngw = 1; ngw <= ng_max; ++ngw) {
                TileGeom t = tile_geom<real>(q.m, q.ell, W, V, ngw, cs);
                if (t.NT > MAX_NT || t.bytes > limit) continue;
                if (t.NG > 1 && t.Rg < 4) continue;
                // per ED cell: the rows of the Wb columns (plus CS NG seed rows of
                // ell products) over the W positions, the selection, threads
                const double rows = 17.0 + 2.0 * cs * t.NG * (double)q.ell / q.R;
                const double sel = 23.0;
                const bool pair = pair_layout(t, limit);
                const double eff = pair ? std::min(1.0, 2.0 * t.NT / 512.0) : (t.NT >= 384 ? 1.0 : t.NT / 384.0);
                const double cl = cs > 1 ? 1.1 : 1.0;  // partner writes and cluster barriers
                // (every column thread computes its V columns: NTc V of them, Wb rounded up)
                out->push_back(TileCand{cl * ((double)(NTc * V) / W * rows + sel) / eff, W, ngw, t, pair});
            }
        }
    }
}

// Layouts chosen by the autotuner (pastila_tune), process-wide, keyed by
// (precision, m, ell, k): tile width and row groups asked.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::tuple<int, int, int, int>> g_tuned;  // W, row groups asked, GS, CS
uint64_t g_tune_gen = 0;  // bumped by every change of the table (captured graphs depend on it)

uint64_t tune_generation() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune_gen;
}

template <typename real>
std::tuple<int, int, int, int> tune_key(const MParams& q) {
    return std::make_tuple((int)sizeof(real), q.m, q.ell, q.k);
}

template <typename real, int V>
pastila_status choose_tile_s(size_t limit, const MParams& q, TileGeom* g, bool clusters = true) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key<real>(q));
        if (it != g_tuned.end() && (clusters || std::get<3>(it->second) == 1)) {
            TileGeom t = tile_geom<real>(q.m, q.ell, std::get<0>(it->second), V, std::get<1>(it->second),
                                         std::get<3>(it->second));
            t.GS = std::get<2>(it->second);
            if (t.NT <= MAX_NT && t.bytes <= limit) {
                *g = t;
                return PASTILA_OK;
            }
        }
    }
    std::vector<TileCand> c;
    tile_candidates<real, V>(limit, q, &c, clusters);
    if (c.empty()) return fail(PASTILA_EINVAL, "m = %d, ell = %d: the tile does not fit in shared memory", q.m, q.ell);
    size_t b = 0;
    for (size_t i = 1; i < c.size(); ++i)
        if (c[i].cost < c[b].cost) b = i;
    *g = c[b].g;
    return PASTILA_OK;
}

template <typename real, int V>
pastila_status choose_tile(const pastila_series* h, const MParams& q, TileGeom* g, bool clusters = true) {
    return choose_tile_s<real, V>((size_t)h->smem_optin, q, g, clusters);
}

pastila_status get_event(pastila_series* h, cudaEvent_t* e) {
    if (!h->ev_free.empty()) {
        *e = h->ev_free.back();
        h->ev_free.pop_back();
        return PASTILA_OK;
    }
    CK(cudaEventCreate(e));
    return PASTILA_OK;
}

pastila_status drain_events(pastila_series* h) {
    for (auto& pr : h->ev_pending) {
        CK(cudaEventSynchronize(pr.second));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
        h->tile_ms += ms;
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pending.clear();
    return PASTILA_OK;
}

__global__ void init_dmax_kernel(unsigned long long* k) { *k = KeyOf<double>::enc(0.0); }
__global__ void dec_dmax_kernel(const unsigned long long* k, double* o) { *o = KeyOf<double>::dec(*k); }

template <typename real, int V>
ProfileArgs<real> profile_args(const pastila_series* h, const MParams& q, const Stats* st, const TileGeom& g,
                               real* D, unsigned long long* dmax) {
    ProfileArgs<real> A{};  // every field zero (M, part: the plain, non-streaming form)
    A.Th = (const real*)h->Th;
    A.Tl = (const real*)h->Tl;
    A.muh = (const real*)st->muh;
    A.mul = (const real*)st->mul;
    A.a = (const real*)st->a;
    A.df = (const real*)st->df;
    A.dg = (const real*)st->dg;
    A.n = h->n;
    A.C = q.C;
    A.P = q.P;
    A.m = q.m;
    A.ell = q.ell;
    A.k = q.k;
    A.R = q.R;
    A.S = q.S;
    A.W = g.W;
    A.ntiles = (int)((q.P + g.W - 1) / g.W);
    A.D = D;
    A.dmax_key = dmax;
    A.err = h->err;
    A.spin_limit = h->spin_limit;
    A.test_timeout = h->test_timeout;
    return A;
}

template <typename real, int V>
pastila_status launch_profiles_t(pastila_series* h, const MParams& q, Stats* st, real* D,
                                 unsigned long long* dmax) {
    TileGeom g;
    TRY(choose_tile<real, V>(h, q, &g));
    ProfileArgs<real> A = profile_args<real, V>(h, q, st, g, D, dmax);
    TRY(ensure_kappa(h, q, st, &A.kappa));
    CK(tile_attrs(profile_tiles_kernel<real, V>, h->smem_optin));
    init_dmax_kernel<<<1, 1, 0, h->stream>>>(dmax);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->timing) {
        TRY(get_event(h, &e0));
        TRY(get_event(h, &e1));
        CK(cudaEventRecord(e0, h->stream));
    }
    CK(launch_tiles(profile_tiles_kernel<real, V>, dim3((unsigned)(A.ntiles * g.CS), (unsigned)q.S), g.NT, g.bytes,
                    h->stream, g.CS, A, g));
    CK(cudaGetLastError());
    h->launches += 2;
    if (h->timing) {
        CK(cudaEventRecord(e1, h->stream));
        h->ev_pending.push_back({e0, e1});
        h->tile_launches += 1;
        h->tile_cells += (double)q.S * A.ntiles * (double)q.R * (double)g.Wb;
    }
    return PASTILA_OK;
}

pastila_status launch_profiles(pastila_series* h, const MParams& q, void* D, unsigned long long* dmax) {
    Stats* st;
    TRY(ensure_stats(h, q.ell, &st));
    if (h->prec == PASTILA_FP64) return launch_profiles_t<double, V_F64>(h, q, st, (double*)D, dmax);
    return launch_profiles_t<float, V_F32>(h, q, st, (float*)D, dmax);
}

// ---------------------------------------------------------------------------
// FP64 re-evaluation of near-tied greedy steps on FP32 handles (batch.cuh,
// batched_select_kernel): per length, (K + REF_NCAND) FP64 rows, S area bounds,
// the contenders' FP64 areas and a D-max word for the FP64 tiles; the state
// words live apart (one array for all lengths, cleared once per search).
constexpr double REF_DRHO = 2e-6;  // the FP32 profiles' accuracy in rho at every cell

inline size_t refine_bytes(const MParams& q, int K) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return up(8 * (size_t)(K + REF_NCAND) * (size_t)q.P) + up(4 * (size_t)q.S) + up(8 * REF_NCAND) + up(8) +
           up((size_t)(REF_NCAND + 1) * (size_t)((q.P + 31) / 32));  // tile flags (FP64 tiles are >= 32 wide)
}

// Fills it's refinement fields from region (refine_bytes) and rst (REF_STATE_INTS
// ints); FP64 statistics and the FP64 tile layout of q.
pastila_status refine_attach(pastila_series* h, const MParams& q, int K, BatchItem<float>* it, char* region,
                             int32_t* rst) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    if (!h->fp64_ties) return PASTILA_OK;  // greedy steps decided on FP32 areas alone
    Stats* st;
    TRY(ensure_stats64(h, q.ell, &st));
    TileGeom g;
    TRY(choose_tile<double, V_F64>(h, q, &g));
    ProfileArgs<double> A{};
    A.Th = (const double*)h->Th64;
    A.Tl = (const double*)h->Tl64;
    A.muh = (const double*)st->muh;
    A.mul = (const double*)st->mul;
    A.a = (const double*)st->a;
    A.df = (const double*)st->df;
    A.dg = (const double*)st->dg;
    A.n = h->n;
    A.C = q.C;
    A.P = q.P;
    A.m = q.m;
    A.ell = q.ell;
    A.k = q.k;
    A.R = q.R;
    A.S = q.S;
    A.W = g.W;
    A.ntiles = (int)((q.P + g.W - 1) / g.W);
    A.err = h->err;
    A.spin_limit = h->spin_limit;
    A.test_timeout = h->test_timeout;
    char* r = region;
    it->rows64 = (double*)r;
    r += up(8 * (size_t)(K + REF_NCAND) * (size_t)q.P);
    it->bound = (float*)r;
    r += up(4 * (size_t)q.S);
    it->cand_area = (double*)r;
    r += up(8 * REF_NCAND);
    A.dmax_key = (unsigned long long*)r;  // the FP64 rows' D max (unused)
    r += up(8);
    it->need = (uint8_t*)r;
    A.D = it->rows64;
    it->A64 = A;
    it->G64 = g;
    it->rst = rst;
    it->bc = (float)(2.2 * q.ell * REF_DRHO);
    return PASTILA_OK;
}

// The K greedy steps of n items (device array d_items, host copies hi) on one
// stream: FP32 areas with their bounds, the choice (FP32, or FP64 for a
// near-tied step), the FP64 rows that needs (one launch per refining item), the
// contenders' FP64 areas, the decision and the curve update.  Returns the
// launch count.
template <typename real>
int enqueue_greedy(cudaStream_t s, const BatchItem<real>* d_items, const std::vector<BatchItem<real>>& hi, int K,
                   int64_t maxS, int64_t maxP, int smem_optin, pastila_status* err) {
    const int n = (int)hi.size();
    const unsigned pb = (unsigned)((maxP + 255) / 256);
    bool any = false;
    for (const auto& it : hi) any |= it.rows64 != nullptr;
    int launches = 0;
    *err = PASTILA_OK;
    if (any) {
        const cudaError_t e = tile_attrs(refine_rows_kernel<V_F64>, smem_optin);
        if (e != cudaSuccess) {
            *err = fail(PASTILA_ECUDA, "greedy refinement set-up: %s", cudaGetErrorString(e));
            return 0;
        }
    }
    for (int t = 0; t < K; ++t) {
        batched_area_kernel<real><<<dim3((unsigned)maxS, n), AREA_THREADS, 0, s>>>(d_items, t);
        if (!any) {
            batched_argmin_kernel<real><<<n, 1024, 0, s>>>(d_items, t);
            if (t + 1 < K) batched_update_kernel<real><<<dim3(pb, n), 256, 0, s>>>(d_items, t);
            launches += t + 1 < K ? 3 : 2;
            continue;
        }
        batched_select_kernel<real><<<n, 1024, 0, s>>>(d_items, t);
        launches += 2;
        if constexpr (std::is_same<real, float>::value) {
            int nt64 = 1;
            for (const auto& it : hi)
                if (it.rows64 && it.A64.ntiles > nt64) nt64 = it.A64.ntiles;
            batched_refine_need_kernel<real><<<dim3((unsigned)nt64, n), NEED_THREADS, 0, s>>>(d_items, t);
            ++launches;
        }
        if constexpr (std::is_same<real, float>::value) {
            for (int i = 0; i < n; ++i) {
                const BatchItem<real>& it = hi[i];
                if (!it.rows64 || t >= it.K) continue;
                const TileGeom& g = it.G64;
                const cudaError_t e = launch_tiles(refine_rows_kernel<V_F64>,
                                                   dim3((unsigned)(it.A64.ntiles * g.CS), (unsigned)(it.K + REF_NCAND)), g.NT,
                                                   g.bytes, s, g.CS, d_items + i, t);
                if (e != cudaSuccess) {
                    *err = fail(PASTILA_ECUDA, "FP64 rows launch: %s", cudaGetErrorString(e));
                    return launches;
                }
                ++launches;
            }
        }
        batched_refine_area_kernel<real><<<dim3(REF_NCAND, n), AREA_THREADS, 0, s>>>(d_items, t);
        batched_choose_update_kernel<real><<<dim3(pb, n), 256, 0, s>>>(d_items, t);
        launches += 2;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) *err = fail(PASTILA_ECUDA, "greedy launches: %s", cudaGetErrorString(e));
    return launches;
}

// Autotuner: times the cost model's layout and its closest rivals (the model's
// best cluster and two-CTA-per-SM layouts, the cheapest of every thread count,
// then by modelled cost within 1.5x of the model's best) on the first min(S, 64)
// segments of this series, and keeps the fastest for (precision, m, ell, k).
template <typename real, int V>
pastila_status tune_t(pastila_series* h, const MParams& q, int max_cand, pastila_tune_result* res) {
    std::vector<TileCand> c;
    tile_candidates<real, V>((size_t)h->smem_optin, q, &c);
    if (c.empty()) return fail(PASTILA_EINVAL, "m = %d, ell = %d: the tile does not fit in shared memory", q.m, q.ell);
    std::stable_sort(c.begin(), c.end(), [](const TileCand& x, const TileCand& y) { return x.cost < y.cost; });
    std::vector<TileCand> pick;
    std::vector<int> nts;
    auto key = [](const TileCand& t) { return t.g.NT * 4 + t.g.CS; };
    pick.push_back(c[0]);  // the model's choice, timed first
    nts.push_back(key(c[0]));
    // the model's best of every cluster size and of the layouts that put two
    // CTAs on an SM are always timed
    auto best_of = [&](auto pred) {
        for (const TileCand& t : c) {
            if (!pred(t)) continue;
            bool have = false;
            for (const TileCand& u : pick) have |= pred(u);
            if (!have && (int)pick.size() < max_cand) {
                pick.push_back(t);
                nts.push_back(key(t));
            }
            return;
        }
    };
    best_of([](const TileCand& t) { return t.g.CS == 2; });
    best_of([](const TileCand& t) { return t.g.CS == 4; });
    best_of([](const TileCand& t) { return t.pair; });
    for (const TileCand& t : c) {  // the cheapest layout of every thread count and cluster size
        if ((int)pick.size() >= max_cand || t.cost > 1.5 * c[0].cost) break;
        if (std::find(nts.begin(), nts.end(), key(t)) == nts.end()) {
            nts.push_back(key(t));
            pick.push_back(t);
        }
    }
    for (const TileCand& t : c) {  // then by modelled cost
        if ((int)pick.size() >= max_cand || t.cost > 1.5 * c[0].cost) break;
        bool have = false;
        for (const TileCand& u : pick) have |= u.W == t.W && u.g.NG == t.g.NG && u.g.CS == t.g.CS;
        if (!have) pick.push_back(t);
    }
    Stats* st;
    TRY(ensure_stats(h, q.ell, &st));
    const int S_sub = q.S < 64 ? q.S : 64;
    void *D, *dk;
    TRY(scratch(h, "tune_D", sizeof(real) * (size_t)S_sub * (size_t)q.P, &D));
    TRY(scratch(h, "tune_dmax", 8, &dk));
    CK(tile_attrs(profile_tiles_kernel<real, V>, h->smem_optin));
    cudaEvent_t e0, e1;
    TRY(get_event(h, &e0));
    TRY(get_event(h, &e1));
    double best_ms = 1e300, model_ms = 0.0;
    size_t bi = 0;
    for (size_t i = 0; i < pick.size(); ++i) {
        const TileGeom& g = pick[i].g;
        ProfileArgs<real> A = profile_args<real, V>(h, q, st, g, (real*)D, (unsigned long long*)dk);
        TRY(ensure_kappa(h, q, st, &A.kappa));
        const dim3 grid((unsigned)(A.ntiles * g.CS), (unsigned)S_sub);
        CK(launch_tiles(profile_tiles_kernel<real, V>, grid, g.NT, g.bytes, h->stream, g.CS, A, g));  // warm-up
        float best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, h->stream));
            CK(launch_tiles(profile_tiles_kernel<real, V>, grid, g.NT, g.bytes, h->stream, g.CS, A, g));
            CK(cudaEventRecord(e1, h->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            best = ms < best ? ms : best;
        }
        CK(cudaGetLastError());
        h->launches += 3;
        if (i == 0) model_ms = best;
        // a rival replaces the layout kept so far only when it is faster by more
        // than TUNE_MARGIN: layouts within timing noise of each other do not
        // trade places from one run to the next (and with them the rounding of
        // the results)
        if (i == 0 || best < best_ms * (1.0 - TUNE_MARGIN)) {
            best_ms = best;
            bi = i;
        }
    }
    h->ev_free.push_back(e0);
    h->ev_free.push_back(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[tune_key<real>(q)] = std::make_tuple(pick[bi].W, pick[bi].ngw, pick[bi].g.GS, pick[bi].g.CS);
        g_tune_gen++;
    }
    if (res) {
        res->m = q.m;
        res->W = pick[bi].g.W;
        res->NG = pick[bi].g.NG;
        res->NT = pick[bi].g.NT;
        res->GS = pick[bi].g.GS;
        res->CS = pick[bi].g.CS;
        res->candidates = (int32_t)pick.size();
        res->ms_model = model_ms;
        res->ms_best = best_ms;
    }
    return PASTILA_OK;
}

// Greedy (eqs. 16-17) + neighbours (eqs. 6-8) on a resident D.  Results stay on
// the device in the named scratch buffers "sn_*"; criterion optional.
template <typename real>
pastila_status snippets_on_device_t(pastila_series* h, const MParams& q, const real* D, int K,
                                    int32_t* labels_dev, const unsigned long long* dmax,
                                    double* crit_dev) {
    void *area, *M, *chosen, *aafter, *counts, *oi, *orank, *ofrac, *oarea, *part;
    TRY(scratch(h, "sn_area", 8 * (size_t)q.S, &area));
    TRY(scratch(h, "sn_M", sizeof(real) * (size_t)q.P, &M));
    TRY(scratch(h, "sn_chosen", 4 * 64, &chosen));
    TRY(scratch(h, "sn_aafter", 8 * 64, &aafter));
    TRY(scratch(h, "sn_counts", 8 * 64, &counts));
    TRY(scratch(h, "sn_oi", 4 * 64, &oi));
    TRY(scratch(h, "sn_orank", 4 * 64, &orank));
    TRY(scratch(h, "sn_ofrac", 8 * 64, &ofrac));
    TRY(scratch(h, "sn_oarea", 8 * 64, &oarea));
    const unsigned pb = (unsigned)((q.P + 255) / 256);
    if constexpr (std::is_same<real, float>::value) {
        // the greedy steps as a one-item batch, with the FP64 re-evaluation of
        // near-tied steps (the same kernels as a select_length sweep)
        void *dit, *rreg, *rst;
        TRY(scratch(h, "sn_item", sizeof(BatchItem<real>), &dit));
        TRY(scratch(h, "sn_refine", refine_bytes(q, K), &rreg));
        TRY(scratch(h, "sn_rst", 4 * REF_STATE_INTS, &rst));
        std::vector<BatchItem<real>> hi(1, BatchItem<real>{});
        BatchItem<real>& it = hi[0];
        it.A.D = const_cast<real*>(D);
        it.A.S = q.S;
        it.A.P = q.P;
        it.A.m = q.m;
        it.M = (real*)M;
        it.area = (double*)area;
        it.chosen = (int32_t*)chosen;
        it.area_after = (double*)aafter;
        it.K = K;
        TRY(refine_attach(h, q, K, &it, (char*)rreg, (int32_t*)rst));
        CK(cudaMemcpyAsync(dit, &it, sizeof(BatchItem<real>), cudaMemcpyHostToDevice, h->stream));
        pastila_status gst;
        h->launches += enqueue_greedy<real>(h->stream, (const BatchItem<real>*)dit, hi, K, q.S, q.P, h->smem_optin,
                                            &gst);
        if (gst != PASTILA_OK) return gst;
        h->launches -= 3 * K - 1;  // counted below with the plain steps
    } else {
        for (int t = 0; t < K; ++t) {
            area_kernel<real><<<q.S, AREA_THREADS, 0, h->stream>>>(D, q.S, q.P, t ? (const real*)M : nullptr,
                                                                   (const int32_t*)chosen, t, (double*)area);
            argmin_area_kernel<<<1, 1024, 0, h->stream>>>((const double*)area, q.S, (int32_t*)chosen,
                                                          (double*)aafter, t);
            if (t + 1 < K)
                update_curve_kernel<real><<<pb, 256, 0, h->stream>>>(D, q.P, (const int32_t*)chosen, t, (real*)M);
        }
    }
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(counts, 0, 8 * 64, h->stream));
    neighbors_kernel<real><<<pb, 256, 0, h->stream>>>(D, q.P, (const int32_t*)chosen, K, labels_dev,
                                                      (unsigned long long*)counts);
    finalize_snippets_kernel<<<1, 1, 0, h->stream>>>((const int32_t*)chosen, (const double*)aafter,
                                                     (const unsigned long long*)counts, K, q.P, (int32_t*)oi,
                                                     (int32_t*)orank, (double*)ofrac, (double*)oarea);
    CK(cudaGetLastError());
    h->launches += 3 * K - 1 + 2;
    if (crit_dev) {
        const int nb = 296;
        TRY(scratch(h, "crit_part", 8 * nb, &part));
        criterion_partial_kernel<real><<<nb, AREA_THREADS, 0, h->stream>>>(D, q.P, (const int32_t*)chosen, K,
                                                                          (double*)part);
        criterion_final_kernel<<<1, 1, 0, h->stream>>>((const double*)part, nb, dmax, crit_dev);
        CK(cudaGetLastError());
        h->launches += 2;
    }
    return PASTILA_OK;
}

pastila_status snippets_on_device(pastila_series* h, const MParams& q, const void* D, int K, int32_t* labels_dev,
                                  const unsigned long long* dmax, double* crit_dev) {
    if (h->prec == PASTILA_FP64)
        return snippets_on_device_t<double>(h, q, (const double*)D, K, labels_dev, dmax, crit_dev);
    return snippets_on_device_t<float>(h, q, (const float*)D, K, labels_dev, dmax, crit_dev);
}

// ---------------------------------------------------------------------------
// Greedy snippet search without the S x P profile set (eqs. 16-17 by lazy
// evaluation), for lengths whose D does not fit.  Rows of D are recomputed by
// the tile kernel; the profiles of the K chosen segments are kept.
//
// Step 0 runs one streaming pass over all segments: every segment's area
// sum_p D_s(p) up to FP64 rounding (relative error far below 1e-9), and a
// sketch of its row over blocks of positions (whole tiles): the block sums and
// the block's largest and smallest value.  The segments whose area lies within
// the rounding margin of the best are recomputed exactly (their rows, then the
// same per-row sum as the materialized path), and the exact minimum wins
// (lowest index on ties).  From step 1 on, every segment's area is bounded from
// below, block by block, by what is known of its row: its block minimum and
// maximum against the current curve M, and, for a row recomputed at an earlier
// step, its block areas then less the block's drop in M since (M only
// shrinks).  Segments are recomputed in order of the bound until the bound
// passes the best exact area.  Every choice and area is therefore the one the
// materialized search makes.
// ---------------------------------------------------------------------------
template <typename real, int V>
pastila_status snippets_streamed_t(pastila_series* h, const MParams& q, int K, int32_t* labels_out,
                                   void* prof_out, int64_t* work) {
    const int S = q.S;
    const int64_t P = q.P;
    const size_t rs = sizeof(real);
    TileGeom g;
    TRY(choose_tile<real, V>(h, q, &g));  // the layout pastila_snippets uses: the same D to the last bit
    Stats* st;
    TRY(ensure_stats(h, q.ell, &st));
    const int ntiles = (int)((P + g.W - 1) / g.W);
    const int CS = g.CS;
    const int ne = ntiles * CS;  // CTA entries per segment: CTA c of tile t covers its positions c Wc ..
    // per-CTA partial sums, maxima and minima of a chunk of segments: <= 256 MiB
    const int chunk = std::max(1, std::min(S, (int)((size_t)(256u << 20) / ((8 + 2 * rs) * (size_t)ne))));
    // position blocks of TB whole tiles (L positions): as fine as 512 MiB of
    // sketches and block areas allow (8 + 8 + 2 rs bytes per segment and block)
    const size_t per_block = (size_t)S * (16 + 2 * rs);
    const int nb_max = (int)std::max<size_t>(1, std::min<size_t>((size_t)ntiles, ((size_t)512 << 20) / per_block));
    const int TB = (ntiles + nb_max - 1) / nb_max, NB = (ntiles + TB - 1) / TB;
    const int64_t L = (int64_t)TB * g.W;
    // rows recomputed per batch: 8 at first, doubling up to BMAX (<= 256 MiB of rows)
    const int BMAX = (int)std::max<int64_t>(8, std::min<int64_t>(32, ((int64_t)256 << 20) / ((int64_t)rs * P)));
    void *part, *pmx, *pmn, *apx, *A0, *Ab, *X, *N, *keep, *M, *rows, *segs, *rarea, *rblk, *dk, *mblk;
    void *Ms, *Mp, *tsd, *tkd, *lbd;
    void *chosen_d, *aafter_d, *counts, *oi, *orank, *ofrac, *oarea, *lab = nullptr;
    TRY(scratch(h, "st_part", 8 * (size_t)chunk * ne, &part));
    TRY(scratch(h, "st_pmx", rs * (size_t)chunk * ne, &pmx));
    TRY(scratch(h, "st_pmn", rs * (size_t)chunk * ne, &pmn));
    TRY(scratch(h, "st_apx", 8 * (size_t)S, &apx));
    TRY(scratch(h, "st_A0", 8 * (size_t)S * NB, &A0));
    TRY(scratch(h, "st_Ab", 8 * (size_t)S * NB, &Ab));
    TRY(scratch(h, "st_X", rs * (size_t)S * NB, &X));
    TRY(scratch(h, "st_N", rs * (size_t)S * NB, &N));
    TRY(scratch(h, "st_keep", rs * (size_t)K * P, &keep));
    TRY(scratch(h, "st_M", rs * (size_t)P, &M));
    TRY(scratch(h, "st_Ms", rs * (size_t)P, &Ms));
    TRY(scratch(h, "st_Mp", 8 * (size_t)P, &Mp));
    TRY(scratch(h, "st_rows", rs * (size_t)BMAX * P, &rows));
    TRY(scratch(h, "st_segs", 4 * (size_t)BMAX, &segs));
    TRY(scratch(h, "st_rarea", 8 * (size_t)BMAX, &rarea));
    TRY(scratch(h, "st_rblk", 8 * (size_t)BMAX * NB, &rblk));
    TRY(scratch(h, "st_ts", 4 * (size_t)S, &tsd));
    TRY(scratch(h, "st_taken", (size_t)S, &tkd));
    TRY(scratch(h, "st_lb", 8 * (size_t)S, &lbd));
    TRY(scratch(h, "dmax", 8, &dk));
    TRY(scratch(h, "st_mblk", 8 * (size_t)(K + 1) * NB, &mblk));
    TRY(scratch(h, "sn_chosen", 4 * 64, &chosen_d));
    TRY(scratch(h, "sn_aafter", 8 * 64, &aafter_d));
    TRY(scratch(h, "sn_counts", 8 * 64, &counts));
    TRY(scratch(h, "sn_oi", 4 * 64, &oi));
    TRY(scratch(h, "sn_orank", 4 * 64, &orank));
    TRY(scratch(h, "sn_ofrac", 8 * 64, &ofrac));
    TRY(scratch(h, "sn_oarea", 8 * 64, &oarea));
    if (labels_out) TRY(scratch(h, "labels", 4 * (size_t)P, &lab));
    CK(tile_attrs(stream_tiles_kernel<real, V>, h->smem_optin));
    CK(tile_attrs(rows_tiles_kernel<real, V>, h->smem_optin));
    init_dmax_kernel<<<1, 1, 0, h->stream>>>((unsigned long long*)dk);
    h->launches += 1;
    ProfileArgs<real> A = profile_args<real, V>(h, q, st, g, nullptr, (unsigned long long*)dk);
    TRY(ensure_kappa(h, q, st, &A.kappa));
    int64_t passes = 0, nrows = 0;
    std::vector<double> hapx(S), hlb(S), ex(BMAX);
    // a streaming pass over every segment with the curve Mc (nullptr: +inf):
    // approximate areas (hapx), their block sums into blocks, and the block
    // sketches X, N (the same at every pass: D does not change)
    auto pass = [&](const real* Mc, double* blocks) -> pastila_status {
        ProfileArgs<real> B = A;
        B.M = Mc;
        B.part = (double*)part;
        B.pmx = (real*)pmx;
        B.pmn = (real*)pmn;
        for (int s0 = 0; s0 < S; s0 += chunk) {
            const int ns = std::min(chunk, S - s0);
            CK(launch_tiles(stream_tiles_kernel<real, V>, dim3((unsigned)ne, (unsigned)ns), g.NT, g.bytes, h->stream,
                            CS, B, g, s0));
            segment_sketch_kernel<real><<<ns, AREA_THREADS, 0, h->stream>>>(
                (const double*)part, (const real*)pmx, (const real*)pmn, ne, TB * CS, NB, blocks + (size_t)s0 * NB,
                (real*)X + (size_t)s0 * NB, (real*)N + (size_t)s0 * NB, (double*)apx + s0);
            h->launches += 2;
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hapx.data(), apx, 8 * (size_t)S, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        passes++;
        return PASTILA_OK;
    };
    TRY(pass(nullptr, (double*)A0));  // step 0: the row sums and the sketches
    // exact areas (the materialized path's per-row sums) and block areas of up to BMAX rows
    auto exact = [&](const std::vector<int32_t>& ss, const real* Mc) -> pastila_status {
        const int nb = (int)ss.size();
        CK(cudaMemcpyAsync(segs, ss.data(), 4 * (size_t)nb, cudaMemcpyHostToDevice, h->stream));
        ProfileArgs<real> B = A;
        B.D = (real*)rows;
        CK(launch_tiles(rows_tiles_kernel<real, V>, dim3((unsigned)ne, (unsigned)nb), g.NT, g.bytes, h->stream, CS, B,
                        g, (const int32_t*)segs));
        row_area_kernel<real><<<nb, AREA_THREADS, 0, h->stream>>>((const real*)rows, P, Mc, (double*)rarea);
        row_blocks_kernel<real><<<dim3((unsigned)NB, (unsigned)nb), AREA_THREADS, 0, h->stream>>>(
            (const real*)rows, P, Mc, L, NB, (double*)rblk);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(ex.data(), rarea, 8 * (size_t)nb, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        h->launches += 3;
        nrows += nb;
        return PASTILA_OK;
    };
    const double REL = 1e-9;  // far above the FP64 rounding of these sums
    std::vector<int32_t> chosen;
    std::vector<double> aafter;
    std::vector<unsigned char> taken(S, 0);
    std::vector<int32_t> ts(S, 0);  // step at which a segment's block areas were last taken (0: only the sketch)
    std::vector<real> hM;
    std::vector<double> hMp;
    std::vector<int32_t> order;
    order.reserve(S);
    for (int t = 0; t < K; ++t) {
        const real* Mc = t ? (const real*)M : nullptr;
        if (t == 0) {
            for (int s = 0; s < S; ++s) hlb[s] = hapx[s] - REL * std::fabs(hapx[s]);
        } else {
            // block sums of M at this step, and M sorted within each block with running sums
            curve_blocks_kernel<real><<<NB, AREA_THREADS, 0, h->stream>>>((const real*)M, P, L,
                                                                         (double*)mblk + (size_t)t * NB);
            CK(cudaGetLastError());
            h->launches += 1;
            hM.resize(P);
            hMp.resize(P);
            CK(cudaMemcpyAsync(hM.data(), M, rs * (size_t)P, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            for (int b = 0; b < NB; ++b) {
                const int64_t p0 = (int64_t)b * L, p1 = std::min(P, p0 + L);
                std::sort(hM.begin() + p0, hM.begin() + p1);
                double run = 0.0;
                for (int64_t p = p0; p < p1; ++p) {
                    run += (double)hM[p];
                    hMp[p] = run;
                }
            }
            CK(cudaMemcpyAsync(Ms, hM.data(), rs * (size_t)P, cudaMemcpyHostToDevice, h->stream));
            CK(cudaMemcpyAsync(Mp, hMp.data(), 8 * (size_t)P, cudaMemcpyHostToDevice, h->stream));
            CK(cudaMemcpyAsync(tsd, ts.data(), 4 * (size_t)S, cudaMemcpyHostToDevice, h->stream));
            CK(cudaMemcpyAsync(tkd, taken.data(), (size_t)S, cudaMemcpyHostToDevice, h->stream));
            stream_bounds_kernel<real><<<S, AREA_THREADS, 0, h->stream>>>(
                (const double*)A0, (const double*)Ab, (const real*)X, (const real*)N, (const int32_t*)tsd,
                (const double*)mblk, t, (const real*)Ms, (const double*)Mp, P, L, NB, (const unsigned char*)tkd, REL,
                (double*)lbd);
            CK(cudaGetLastError());
            h->launches += 1;
            CK(cudaMemcpyAsync(hlb.data(), lbd, 8 * (size_t)S, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
        order.clear();
        for (int s = 0; s < S; ++s)
            if (!taken[s]) order.push_back(s);
        auto by_bound = [&](int32_t x, int32_t y) { return hlb[x] < hlb[y] || (hlb[x] == hlb[y] && x < y); };
        std::sort(order.begin(), order.end(), by_bound);
        double best = std::numeric_limits<double>::infinity();
        int32_t bs = -1;
        size_t i = 0;
        int bsz = 8;
        bool passed = t == 0;  // step 0 had its pass
        std::vector<int32_t> batch;
        while (i < order.size() && hlb[order[i]] <= best) {
            batch.clear();
            while (i < order.size() && (int)batch.size() < bsz && hlb[order[i]] <= best) batch.push_back(order[i++]);
            TRY(exact(batch, Mc));
            bsz = std::min(2 * bsz, BMAX);
            for (int j = 0; j < (int)batch.size(); ++j) {
                const int32_t s = batch[j];
                const double ar = ex[j];
                if (t >= 1) {  // this row's block areas at step t, for the later bounds
                    CK(cudaMemcpyAsync((double*)Ab + (size_t)s * NB, (const double*)rblk + (size_t)j * NB,
                                       8 * (size_t)NB, cudaMemcpyDeviceToDevice, h->stream));
                    ts[s] = t;
                }
                hlb[s] = std::numeric_limits<double>::infinity();  // settled at this step
                if (ar < best || (ar == best && s < bs)) {
                    best = ar;
                    bs = s;
                    CK(cudaMemcpyAsync((char*)keep + rs * (size_t)t * P, (const char*)rows + rs * (size_t)j * P,
                                       rs * (size_t)P, cudaMemcpyDeviceToDevice, h->stream));
                }
            }
            // when the bounds leave more than half of the segments open, one pass
            // over all of them costs less than recomputing those rows one by one:
            // it gives every area up to rounding and every block area at step t
            if (!passed) {
                size_t open = 0;
                for (size_t u = i; u < order.size() && hlb[order[u]] <= best; ++u) ++open;
                if (2 * open > (size_t)S) {
                    TRY(pass(Mc, (double*)Ab));
                    passed = true;
                    for (int s = 0; s < S; ++s) {
                        if (taken[s]) continue;
                        ts[s] = t;
                        if (std::isfinite(hlb[s])) hlb[s] = hapx[s] - REL * std::fabs(hapx[s]);
                    }
                    std::vector<int32_t> rest(order.begin() + i, order.end());
                    std::sort(rest.begin(), rest.end(), by_bound);
                    order.swap(rest);
                    i = 0;
                }
            }
        }
        chosen.push_back(bs);
        aafter.push_back(best);
        taken[bs] = 1;
        min_curve_kernel<real><<<(unsigned)((P + 255) / 256), 256, 0, h->stream>>>(
            (const real*)keep + (size_t)t * P, P, t == 0 ? 1 : 0, (real*)M);
        CK(cudaGetLastError());
        h->launches += 1;
    }
    CK(cudaMemcpyAsync(chosen_d, chosen.data(), 4 * (size_t)K, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(aafter_d, aafter.data(), 8 * (size_t)K, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(counts, 0, 8 * 64, h->stream));
    neighbors_rows_kernel<real><<<(unsigned)((P + 255) / 256), 256, 0, h->stream>>>(
        (const real*)keep, P, (const int32_t*)chosen_d, K, (int32_t*)lab, (unsigned long long*)counts);
    finalize_snippets_kernel<<<1, 1, 0, h->stream>>>((const int32_t*)chosen_d, (const double*)aafter_d,
                                                     (const unsigned long long*)counts, K, P, (int32_t*)oi,
                                                     (int32_t*)orank, (double*)ofrac, (double*)oarea);
    CK(cudaGetLastError());
    h->launches += 2;
    if (labels_out) CK(cudaMemcpyAsync(labels_out, lab, 4 * (size_t)P, cudaMemcpyDeviceToHost, h->stream));
    if (prof_out) CK(cudaMemcpyAsync(prof_out, keep, rs * (size_t)K * P, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (work) {
        work[0] = passes;
        work[1] = nrows;
    }
    return PASTILA_OK;
}

pastila_status streamed(pastila_series* h, const MParams& q, int K, int32_t* labels_out, void* prof_out,
                        int64_t* work) {
    if (h->prec == PASTILA_FP64) return snippets_streamed_t<double, V_F64>(h, q, K, labels_out, prof_out, work);
    return snippets_streamed_t<float, V_F32>(h, q, K, labels_out, prof_out, work);
}

pastila_status read_snippets(pastila_series* h, int K, pastila_snippet* out) {
    std::vector<int32_t> oi(K), orank(K);
    std::vector<double> ofrac(K), oarea(K);
    CK(cudaMemcpyAsync(oi.data(), h->bufs["sn_oi"].p, 4 * K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(orank.data(), h->bufs["sn_orank"].p, 4 * K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(ofrac.data(), h->bufs["sn_ofrac"].p, 8 * K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(oarea.data(), h->bufs["sn_oarea"].p, 8 * K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < K; ++i) {
        out[i].index = oi[i];
        out[i].rank = orank[i];
        out[i].frac = ofrac[i];
        out[i].area_after = oarea[i];
    }
    return PASTILA_OK;
}

// ---------------------------------------------------------------------------
// The whole length sweep of select_length in batched launches (FP32 handles):
// statistics for every distinct ell, one tile launch for all lengths, the greedy
// steps, the eq. 18 criterion and m_best, and the eq. 8 records of m_best, with
// no host synchronisation in between (so the sequence can be captured in a CUDA
// graph and replayed).
// ---------------------------------------------------------------------------
// One tile launch of a sweep: the lengths whose tiles use clusters of cs CTAs
// (a launch has a single cluster shape), as items [first, first + n) of the
// tile-item array, with their own CTA numbering.
struct TileGroup {
    int cs = 1, first = 0, n = 0, block = 0;
    size_t smem = 0;
    long long ctas = 0;
};

struct SweepBufs {
    std::vector<TileGroup> groups;
    void* tiles = nullptr;  // tile items, grouped by cluster size
    void* items = nullptr;
    void* best = nullptr;
    void* counts = nullptr;
    void* rec_index = nullptr;
    void* rec_rank = nullptr;
    void* rec_frac = nullptr;
    void* rec_area = nullptr;
    void* crit = nullptr;
    void* rst = nullptr;  // refinement state words, REF_STATE_INTS per item
};

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename real, int V>
pastila_status sweep_prepare_t(pastila_series* h, const std::vector<MParams>& qs, int K, SweepBufs* sb,
                               std::vector<BatchItem<real>>* items_out, std::vector<BatchItem<real>>* tiles_out,
                               int64_t* maxS_out, int64_t* maxP_out) {
    const int n = (int)qs.size();
    std::vector<TileGeom> geo(n);
    for (int i = 0; i < n; ++i) TRY(choose_tile<real, V>(h, qs[i], &geo[i]));
    // one region for every item's D, curve and small arrays
    size_t dbytes = 0, sbytes = 0;
    for (int i = 0; i < n; ++i) {
        dbytes += up256(sizeof(real) * (size_t)qs[i].S * (size_t)qs[i].P);
        sbytes += up256(sizeof(real) * (size_t)qs[i].P) + up256(8 * (size_t)qs[i].S) + up256(4 * 64) +
                  up256(8 * 64) + up256(8 * CRIT_BLOCKS) + up256(8) + up256(8);
    }
    void *dreg, *sreg;
    TRY(scratch(h, "sweep_D", dbytes, &dreg));
    TRY(scratch(h, "sweep_small", sbytes, &sreg));
    TRY(scratch(h, "sweep_items", sizeof(BatchItem<real>) * (size_t)n, &sb->items));
    TRY(scratch(h, "sweep_tiles", sizeof(BatchItem<real>) * (size_t)n, &sb->tiles));
    TRY(scratch(h, "sweep_best", 16, &sb->best));
    TRY(scratch(h, "sweep_counts", 8 * 64, &sb->counts));
    TRY(scratch(h, "sweep_rec_index", 4 * 64, &sb->rec_index));
    TRY(scratch(h, "sweep_rec_rank", 4 * 64, &sb->rec_rank));
    TRY(scratch(h, "sweep_rec_frac", 8 * 64, &sb->rec_frac));
    TRY(scratch(h, "sweep_rec_area", 8 * 64, &sb->rec_area));
    // FP64 re-evaluation of near-tied greedy steps (FP32 handles)
    constexpr bool refine = std::is_same<real, float>::value;
    void* rreg = nullptr;
    if (refine) {
        size_t rbytes = 0;
        for (int i = 0; i < n; ++i) rbytes += refine_bytes(qs[i], K);
        TRY(scratch(h, "sweep_refine", rbytes, &rreg));
        TRY(scratch(h, "sweep_rst", 4 * (size_t)n * REF_STATE_INTS, &sb->rst));
    }
    std::vector<Stats*> st(n);
    for (int i = 0; i < n; ++i) TRY(ensure_stats(h, qs[i].ell, &st[i]));
    std::vector<BatchItem<real>>& items = *items_out;
    items.assign(n, BatchItem<real>{});
    char* dp = (char*)dreg;
    char* sp = (char*)sreg;
    int64_t maxS = 0, maxP = 0;
    for (int i = 0; i < n; ++i) {
        const MParams& q = qs[i];
        BatchItem<real>& it = items[i];
        it.A = profile_args<real, V>(h, q, st[i], geo[i], (real*)dp, nullptr);  // D max key below
        TRY(ensure_kappa(h, q, st[i], &it.A.kappa));
        ProfileArgs<real>& A = it.A;
        dp += up256(sizeof(real) * (size_t)q.S * (size_t)q.P);
        it.G = geo[i];
        it.ctas = (long long)q.S * A.ntiles * geo[i].CS;
        it.M = (real*)sp;
        sp += up256(sizeof(real) * (size_t)q.P);
        it.area = (double*)sp;
        sp += up256(8 * (size_t)q.S);
        it.chosen = (int32_t*)sp;
        sp += up256(4 * 64);
        it.area_after = (double*)sp;
        sp += up256(8 * 64);
        it.crit_part = (double*)sp;
        sp += up256(8 * CRIT_BLOCKS);
        it.crit = (double*)sp;
        sp += up256(8);
        A.dmax_key = (unsigned long long*)sp;
        sp += up256(8);
        it.K = K;
        if constexpr (refine) {
            TRY(refine_attach(h, q, K, &it, (char*)rreg, (int32_t*)sb->rst + (size_t)i * REF_STATE_INTS));
            rreg = (char*)rreg + refine_bytes(q, K);
        }
        maxS = q.S > maxS ? q.S : maxS;
        maxP = q.P > maxP ? q.P : maxP;
    }
    // tile launches: one per cluster size, and apart the layouts that put two
    // CTAs on an SM; each numbers its own CTAs (counts are multiples of the
    // cluster size, so every item starts a cluster)
    std::vector<BatchItem<real>>& tiles = *tiles_out;
    tiles.clear();
    sb->groups.clear();
    for (int cls = 0; cls < 6; ++cls) {
        const int cs = 1 << (cls >> 1);
        const bool pair = cls & 1;
        TileGroup tg;
        tg.cs = cs;
        tg.first = (int)tiles.size();
        for (int i = 0; i < n; ++i) {
            if (geo[i].CS != cs || pair_layout(geo[i], (size_t)h->smem_optin) != pair) continue;
            BatchItem<real> t = items[i];
            t.cta_begin = tg.ctas;
            tg.ctas += t.ctas;
            tg.block = geo[i].NT > tg.block ? geo[i].NT : tg.block;
            tg.smem = geo[i].bytes > tg.smem ? geo[i].bytes : tg.smem;
            tiles.push_back(t);
        }
        tg.n = (int)tiles.size() - tg.first;
        if (tg.n) sb->groups.push_back(tg);
    }
    *maxS_out = maxS;
    *maxP_out = maxP;
    return PASTILA_OK;
}

// The launches of one sweep on the handle's stream.  Statistics are recomputed
// for every distinct ell (the series may have been reloaded).
// phase 0: statistics and D-max reset; phase 1: the tile launch; phase 2: the
// greedy steps, the criterion, m_best and its eq. 8 records
template <typename real, int V>
pastila_status sweep_enqueue_t(pastila_series* h, const std::vector<MParams>& qs, int K, const SweepBufs& sb,
                               const std::vector<BatchItem<real>>& hitems, int64_t maxS, int64_t maxP, int phase) {
    const int n = (int)qs.size();
    const BatchItem<real>* items = (const BatchItem<real>*)sb.items;
    if (phase == 1) {
        // the attribute is process-wide: every caller sets the same device maximum, so
        // concurrent callers (handles, the engine) never lower it under one another
        CK(tile_attrs(batched_tiles_kernel<real, V>, h->smem_optin));
        for (const TileGroup& tg : sb.groups) {
            CK(launch_tiles(batched_tiles_kernel<real, V>, dim3((unsigned)tg.ctas), tg.block, tg.smem, h->stream,
                            tg.cs, (const BatchItem<real>*)sb.tiles + tg.first, tg.n));
            h->launches += 1;
        }
        CK(cudaGetLastError());
        return PASTILA_OK;
    }
    if (phase == 2) {
        const unsigned pb = (unsigned)((maxP + 255) / 256);
        pastila_status gst;
        const int gl = enqueue_greedy<real>(h->stream, items, hitems, K, maxS, maxP, h->smem_optin, &gst);
        if (gst != PASTILA_OK) return gst;
        batched_criterion_kernel<real><<<dim3(CRIT_BLOCKS, n), AREA_THREADS, 0, h->stream>>>(items);
        batched_finish_kernel<real><<<1, 256, 0, h->stream>>>(items, n, (int32_t*)sb.best);
        CK(cudaMemsetAsync(sb.counts, 0, 8 * 64, h->stream));
        batched_neighbors_kernel<real><<<pb, 256, 0, h->stream>>>(items, (const int32_t*)sb.best, nullptr,
                                                                  (unsigned long long*)sb.counts);
        batched_records_kernel<real><<<1, 1, 0, h->stream>>>(items, (const int32_t*)sb.best,
                                                             (const unsigned long long*)sb.counts,
                                                             (int32_t*)sb.rec_index, (int32_t*)sb.rec_rank,
                                                             (double*)sb.rec_frac, (double*)sb.rec_area);
        CK(cudaGetLastError());
        h->launches += gl + 4;
        h->phase2_launches = gl + 4;
        return PASTILA_OK;
    }
    std::vector<int> done_ell;
    for (int i = 0; i < n; ++i) {
        bool seen = false;
        for (int e : done_ell) seen |= e == qs[i].ell;
        if (seen) continue;
        done_ell.push_back(qs[i].ell);
        // recompute every statistic in place (find, not operator[]: an entry the
        // map does not hold yet would be created with null buffers)
        auto f = h->stats.find(qs[i].ell);
        if (f != h->stats.end()) f->second.stale = true;
        Stats* st;
        TRY(ensure_stats(h, qs[i].ell, &st));
        if (std::is_same<real, float>::value && h->fp64_ties) {  // the greedy re-evaluation's FP64 statistics
            auto f64 = h->stats64.find(qs[i].ell);
            if (f64 != h->stats64.end()) f64->second.stale = true;
            TRY(ensure_stats64(h, qs[i].ell, &st));
        }
    }
    for (int i = 0; i < n; ++i) {  // the FP32 tiles' conditioning ratios, from the new statistics
        const float* kp;
        TRY(ensure_kappa(h, qs[i], &h->stats[qs[i].ell], &kp));
    }
    batched_init_dmax_kernel<real><<<1, 64, 0, h->stream>>>(items, n);
    CK(cudaGetLastError());
    h->launches += 1;
    return PASTILA_OK;
}

// The profile sets of several lengths from the sweep's batched tile launch (FP32
// handles): the sweep's items with each D pointing at the caller's buffer, then
// its statistics phase and its tile phase, and each length's D maximum decoded.
template <typename real, int V>
pastila_status profiles_batch_t(pastila_series* h, const std::vector<MParams>& qs, void* const* D_dev,
                                double* D_max_dev) {
    SweepBufs sb;
    std::vector<BatchItem<real>> items, tiles;
    int64_t maxS, maxP;
    TRY(sweep_prepare_t<real, V>(h, qs, 2, &sb, &items, &tiles, &maxS, &maxP));
    const int n = (int)qs.size();
    for (BatchItem<real>& t : tiles)
        for (int i = 0; i < n; ++i)
            if (t.A.D == items[i].A.D) t.A.D = (real*)D_dev[i];
    for (int i = 0; i < n; ++i) items[i].A.D = (real*)D_dev[i];
    CK(cudaMemcpyAsync(sb.items, items.data(), sizeof(BatchItem<real>) * items.size(), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemcpyAsync(sb.tiles, tiles.data(), sizeof(BatchItem<real>) * tiles.size(), cudaMemcpyHostToDevice,
                       h->stream));
    {
        NvtxRange range("pastila: window statistics");
        TRY(sweep_enqueue_t<real, V>(h, qs, 2, sb, items, maxS, maxP, 0));
    }
    {
        NvtxRange range("pastila: profile tiles");
        TRY(sweep_enqueue_t<real, V>(h, qs, 2, sb, items, maxS, maxP, 1));
    }
    if (D_max_dev) {
        for (int i = 0; i < n; ++i)
            dec_dmax_kernel<<<1, 1, 0, h->stream>>>(items[i].A.dmax_key, D_max_dev + i);
        CK(cudaGetLastError());
        h->launches += (uint64_t)n;
    }
    return PASTILA_OK;
}

// select_length on FP32 handles: batched, captured into a CUDA graph on the
// second call with the same configuration and replayed from then on.
template <typename real, int V>
pastila_status select_length_batched_t(pastila_series* h, const int32_t* m_list, int n_m, pastila_mparams rule,
                                       const std::vector<MParams>& qs, int K, int32_t* m_best, double* crit_out,
                                       pastila_snippet* best_out) {
    SweepBufs sb;
    std::vector<BatchItem<real>> items, tiles;
    int64_t maxS, maxP;
    TRY(sweep_prepare_t<real, V>(h, qs, K, &sb, &items, &tiles, &maxS, &maxP));
    CK(cudaMemcpyAsync(sb.items, items.data(), sizeof(BatchItem<real>) * items.size(), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemcpyAsync(sb.tiles, tiles.data(), sizeof(BatchItem<real>) * tiles.size(), cudaMemcpyHostToDevice,
                       h->stream));
    auto& gr = h->graph;
    double cells = 0.0;  // ED cells of the tile launch, halo columns included
    for (int i = 0; i < n_m; ++i) {
        const TileGeom& g = items[i].G;
        cells += (double)qs[i].S * (double)items[i].A.ntiles * (double)qs[i].R * (double)g.Wb;
    }
    const uint64_t tgen = tune_generation();
    const bool same = gr.ms == std::vector<int32_t>(m_list, m_list + n_m) && gr.rule.ell == rule.ell &&
                      gr.rule.k == rule.k && gr.K == K && gr.gen == h->alloc_gen && gr.tune_gen == tgen;
    if (!same) {
        for (auto& e : gr.exec)
            if (e) cudaGraphExecDestroy(e);
        gr.exec[0] = gr.exec[1] = gr.exec[2] = nullptr;
        gr.ms.assign(m_list, m_list + n_m);
        gr.rule = rule;
        gr.K = K;
        gr.gen = h->alloc_gen;
        gr.tune_gen = tgen;
        gr.calls = 0;
    }
    gr.calls++;
    if (!gr.ev0) {
        CK(cudaEventCreate(&gr.ev0));
        CK(cudaEventCreate(&gr.ev1));
    }
    if (!gr.exec[0] && gr.calls >= 2) {  // capture the three phases
        const uint64_t l0 = h->launches;
        for (int ph = 0; ph < 3; ++ph) {
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            pastila_status st = sweep_enqueue_t<real, V>(h, qs, K, sb, items, maxS, maxP, ph);
            cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
            if (st != PASTILA_OK) return st;
            if (ec != cudaSuccess) return fail(PASTILA_ECUDA, "graph capture: %s", cudaGetErrorString(ec));
            cudaError_t ei = cudaGraphInstantiate(&gr.exec[ph], graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) return fail(PASTILA_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
        }
        h->launches = l0;
        gr.gen = h->alloc_gen;
    }
    const uint64_t l_before = h->launches;
    static const char* const phase_name[3] = {"pastila: window statistics", "pastila: profile tiles",
                                              "pastila: greedy snippets and length criterion"};
    for (int ph = 0; ph < 3; ++ph) {
        NvtxRange range(phase_name[ph]);
        if (ph == 1 && h->timing) CK(cudaEventRecord(gr.ev0, h->stream));
        if (gr.exec[ph]) {
            CK(cudaGraphLaunch(gr.exec[ph], h->stream));
        } else {
            TRY(sweep_enqueue_t<real, V>(h, qs, K, sb, items, maxS, maxP, ph));
        }
        if (ph == 1 && h->timing) CK(cudaEventRecord(gr.ev1, h->stream));
    }
    if (gr.exec[0]) {  // graph replays: the launches the three captured phases hold
        uint64_t nst = 0;
        std::vector<int> seen;
        for (const MParams& q : qs)
            if (std::find(seen.begin(), seen.end(), q.ell) == seen.end()) seen.push_back(q.ell);
        nst = (std::is_same<real, float>::value && h->fp64_ties ? 4 : 2) * (uint64_t)seen.size();
        if (std::is_same<real, float>::value) nst += (uint64_t)n_m;  // conditioning ratios
        h->launches = l_before + nst + 1 + sb.groups.size() + (uint64_t)h->phase2_launches;
    }
    gr.gen = h->alloc_gen;
    int32_t b = 0;
    std::vector<double> cv(n_m);
    std::vector<int32_t> ri(K), rr(K);
    std::vector<double> rf(K), ra(K);
    CK(cudaMemcpyAsync(&b, sb.best, 4, cudaMemcpyDeviceToHost, h->stream));
    for (int i = 0; i < n_m; ++i)
        CK(cudaMemcpyAsync(&cv[i], items[i].crit, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(ri.data(), sb.rec_index, 4 * K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(rr.data(), sb.rec_rank, 4 * K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(rf.data(), sb.rec_frac, 8 * K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(ra.data(), sb.rec_area, 8 * K, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->timing) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, gr.ev0, gr.ev1));
        h->tile_ms += ms;
        h->tile_launches += 1;
        h->tile_cells += cells;
    }
    *m_best = m_list[b];
    if (crit_out) memcpy(crit_out, cv.data(), 8 * (size_t)n_m);
    if (best_out)
        for (int i = 0; i < K; ++i) best_out[i] = pastila_snippet{ri[i], rr[i], rf[i], ra[i]};
    return PASTILA_OK;
}

pastila_status create_common(pastila_series** out, int64_t n, int device, size_t budget,
                             pastila_precision prec, cudaStream_t stream, pastila_series** hp) {
    if (!out) return fail(PASTILA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 4) return fail(PASTILA_EINVAL, "n = %lld: the series needs at least 4 values", (long long)n);
    if (prec != PASTILA_FP32 && prec != PASTILA_FP64) return fail(PASTILA_EINVAL, "unknown precision %d", (int)prec);
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(PASTILA_EINVAL, "device %d: %d device(s) visible", device, ndev);
    CK(cudaSetDevice(device));
    int smem = 0;
    CK(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    pastila_series* h = new pastila_series();
    h->device = device;
    h->prec = prec;
    h->n = n;
    h->budget = budget;
    h->smem_optin = smem - 1024;  // headroom for static shared memory
    if (stream) {
        h->stream = stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return fail(PASTILA_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        h->own_stream = true;
    }
    wait_knobs(&h->spin_limit, &h->test_timeout);
    if (cudaHostAlloc((void**)&h->err, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return fail(PASTILA_ENOMEM, "the handle's error flag could not be allocated");
    }
    *h->err = 0;
    pastila_status st = dev_alloc(h, (void**)&h->T, 8 * (size_t)n);
    if (st != PASTILA_OK) {
        if (h->own_stream) cudaStreamDestroy(h->stream);
        delete h;
        return st;
    }
    *hp = h;
    return PASTILA_OK;
}

pastila_status check_finite(const double* T, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(T[i])) return fail(PASTILA_EINVAL, "T[%lld] is not finite", (long long)i);
    return PASTILA_OK;
}

}  // namespace

#include "engine.cuh"

extern "C" {

const char* pastila_last_error(void) { return g_err.c_str(); }

pastila_status pastila_tune(pastila_series* h, const int32_t* m_list, int32_t n_m, pastila_mparams rule,
                            int32_t max_candidates, pastila_tune_result* out) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    if (!m_list || n_m < 1) return fail(PASTILA_EINVAL, "m_list is empty");
    if (max_candidates < 1 || max_candidates > 64)
        return fail(PASTILA_EINVAL, "max_candidates = %d: must be in [1, 64]", max_candidates);
    TRY(set_device(h));
    for (int i = 0; i < n_m; ++i) {
        MParams q;
        TRY(resolve(h, m_list[i], rule, &q));
        if (h->prec == PASTILA_FP64)
            TRY(tune_t<double, V_F64>(h, q, max_candidates, out ? out + i : nullptr));
        else
            TRY(tune_t<float, V_F32>(h, q, max_candidates, out ? out + i : nullptr));
    }
    return stage_check(h);
}

pastila_status pastila_tune_set(pastila_precision prec, int32_t m, int32_t ell, int32_t k, int32_t W, int32_t NG,
                                int32_t GS, int32_t CS) {
    g_err.clear();
    if (prec != PASTILA_FP32 && prec != PASTILA_FP64) return fail(PASTILA_EINVAL, "unknown precision %d", (int)prec);
    if (m < 4 || ell < 2 || ell > m || k < 1) return fail(PASTILA_EINVAL, "m = %d, ell = %d, k = %d out of range", m, ell, k);
    if (W < 32 || W % 32) return fail(PASTILA_EINVAL, "W = %d: a positive multiple of 32", W);
    if (NG < 1 || NG > 64) return fail(PASTILA_EINVAL, "NG = %d: 1 .. 64 row groups", NG);
    if (GS != 32) return fail(PASTILA_EINVAL, "GS = %d: the selection runs one warp (32 lanes) per run", GS);
    if (CS != 1 && CS != 2 && CS != 4) return fail(PASTILA_EINVAL, "CS = %d: 1, 2 or 4", CS);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_tuple(prec == PASTILA_FP64 ? 8 : 4, m, ell, k)] = std::make_tuple(W, NG, GS, CS);
    g_tune_gen++;
    return PASTILA_OK;
}

pastila_status pastila_tune_get(pastila_precision prec, int32_t m, int32_t ell, int32_t k, int32_t* W, int32_t* NG,
                                int32_t* GS, int32_t* CS) {
    g_err.clear();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(prec == PASTILA_FP64 ? 8 : 4, m, ell, k));
    if (it == g_tuned.end()) return fail(PASTILA_EINVAL, "no tuned layout for m = %d, ell = %d, k = %d", m, ell, k);
    if (W) *W = std::get<0>(it->second);
    if (NG) *NG = std::get<1>(it->second);
    if (GS) *GS = std::get<2>(it->second);
    if (CS) *CS = std::get<3>(it->second);
    return PASTILA_OK;
}

pastila_status pastila_plan_layout(pastila_precision prec, int64_t n, int32_t m, pastila_mparams mp,
                                   size_t smem_limit, int32_t* out8) {
    g_err.clear();
    if (!out8) return fail(PASTILA_EINVAL, "out is NULL");
    if (prec != PASTILA_FP32 && prec != PASTILA_FP64) return fail(PASTILA_EINVAL, "unknown precision %d", (int)prec);
    MParams q;
    TRY(resolve_n(n, m, mp, &q));
    TileGeom g;
    if (prec == PASTILA_FP64)
        TRY(choose_tile_s<double, V_F64>(smem_limit, q, &g));
    else
        TRY(choose_tile_s<float, V_F32>(smem_limit, q, &g));
    const int32_t v[8] = {g.W, g.NG, g.NT, g.GS, g.CS, g.Rg, g.Rh, (int32_t)g.bytes};
    memcpy(out8, v, sizeof v);
    return PASTILA_OK;
}

pastila_status pastila_tile_layout(pastila_series* h, int32_t m, pastila_mparams mp, int32_t* out5) {
    g_err.clear();
    if (!h || !out5) return fail(PASTILA_EINVAL, "handle or out is NULL");
    MParams q;
    TRY(resolve(h, m, mp, &q));
    TileGeom g;
    if (h->prec == PASTILA_FP64)
        TRY(choose_tile<double, V_F64>(h, q, &g));
    else
        TRY(choose_tile<float, V_F32>(h, q, &g));
    out5[0] = g.W;
    out5[1] = g.NG;
    out5[2] = g.NT;
    out5[3] = g.GS;
    out5[4] = g.CS;
    return PASTILA_OK;
}

void pastila_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    g_tune_gen++;
}

pastila_status pastila_create(pastila_series** out, const double* T, int64_t n, int device,
                              size_t mem_budget_bytes, pastila_precision prec) {
    g_err.clear();
    if (!T) return fail(PASTILA_EINVAL, "T is NULL");
    if (!out) return fail(PASTILA_EINVAL, "out is NULL");
    TRY(check_finite(T, n));
    pastila_series* h = nullptr;
    TRY(create_common(out, n, device, mem_budget_bytes, prec, nullptr, &h));
    cudaError_t e = cudaMemcpyAsync(h->T, T, 8 * (size_t)n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        pastila_destroy(h);
        return fail(PASTILA_ECUDA, "copying T: %s", cudaGetErrorString(e));
    }
    *out = h;
    return PASTILA_OK;
}

pastila_status pastila_create_device(pastila_series** out, const double* T_dev, int64_t n, int device,
                                     size_t mem_budget_bytes, pastila_precision prec, void* stream) {
    g_err.clear();
    if (!T_dev) return fail(PASTILA_EINVAL, "T_dev is NULL");
    pastila_series* h = nullptr;
    TRY(create_common(out, n, device, mem_budget_bytes, prec, (cudaStream_t)stream, &h));
    cudaError_t e = cudaMemcpyAsync(h->T, T_dev, 8 * (size_t)n, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) {
        pastila_destroy(h);
        return fail(PASTILA_ECUDA, "copying T: %s", cudaGetErrorString(e));
    }
    *out = h;
    return PASTILA_OK;
}

pastila_status pastila_reload(pastila_series* h, const double* T) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    if (!T) return fail(PASTILA_EINVAL, "T is NULL");
    TRY(check_finite(T, h->n));
    TRY(set_device(h));
    CK(cudaMemcpyAsync(h->T, T, 8 * (size_t)h->n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    invalidate_stats(h);
    return PASTILA_OK;
}

pastila_status pastila_reload_device(pastila_series* h, const double* T_dev) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    if (!T_dev) return fail(PASTILA_EINVAL, "T_dev is NULL");
    TRY(set_device(h));
    CK(cudaMemcpyAsync(h->T, T_dev, 8 * (size_t)h->n, cudaMemcpyDeviceToDevice, h->stream));
    invalidate_stats(h);
    return PASTILA_OK;
}

void pastila_destroy(pastila_series* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    for (auto& pr : h->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto e : h->ev_free) cudaEventDestroy(e);
    for (auto& e : h->graph.exec)
        if (e) cudaGraphExecDestroy(e);
    if (h->graph.ev0) cudaEventDestroy(h->graph.ev0);
    if (h->graph.ev1) cudaEventDestroy(h->graph.ev1);
    for (auto& kv : h->stats) {
        cudaFree(kv.second.mu);
        cudaFree(kv.second.a);
        cudaFree(kv.second.df);
        cudaFree(kv.second.dg);
        cudaFree(kv.second.muh);
        cudaFree(kv.second.mul);
    }
    for (auto& kv : h->stats64) {
        cudaFree(kv.second.mu);
        cudaFree(kv.second.a);
        cudaFree(kv.second.df);
        cudaFree(kv.second.dg);
        cudaFree(kv.second.muh);
        cudaFree(kv.second.mul);
    }
    for (auto& kv : h->bufs) cudaFree(kv.second.p);
    cudaFree(h->T);
    cudaFree(h->Th);
    cudaFree(h->Tl);
    cudaFree(h->Th64);
    cudaFree(h->Tl64);
    if (h->err) cudaFreeHost(h->err);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

uint64_t pastila_kernel_launches(const pastila_series* h) { return h ? h->launches : 0; }

pastila_status pastila_set_timing(pastila_series* h, int on) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    TRY(set_device(h));
    TRY(drain_events(h));
    h->timing = on != 0;
    h->tile_ms = 0.0;
    h->tile_launches = 0;
    h->tile_cells = 0.0;
    return PASTILA_OK;
}

pastila_status pastila_tile_time(pastila_series* h, double* ms, int64_t* launches, double* ed_cells) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    TRY(set_device(h));
    TRY(drain_events(h));
    if (ms) *ms = h->tile_ms;
    if (launches) *launches = h->tile_launches;
    if (ed_cells) *ed_cells = h->tile_cells;
    return PASTILA_OK;
}

pastila_status pastila_profiles_device(pastila_series* h, int32_t m, pastila_mparams mp, void* D_dev,
                                       double* D_max_dev) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    if (!D_dev) return fail(PASTILA_EINVAL, "D_dev is NULL");
    TRY(set_device(h));
    MParams q;
    TRY(resolve(h, m, mp, &q));
    void* dk;
    TRY(scratch(h, "dmax", 8, &dk));
    TRY(launch_profiles(h, q, D_dev, (unsigned long long*)dk));
    if (D_max_dev) {
        dec_dmax_kernel<<<1, 1, 0, h->stream>>>((const unsigned long long*)dk, D_max_dev);
        CK(cudaGetLastError());
        h->launches += 1;
    }
    return PASTILA_OK;
}

pastila_status pastila_profiles_batch_device(pastila_series* h, const int32_t* m_list, int32_t n_m,
                                             pastila_mparams rule, void* const* D_dev, double* D_max_dev) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    if (!m_list || n_m < 1) return fail(PASTILA_EINVAL, "m_list is empty");
    if (!D_dev) return fail(PASTILA_EINVAL, "D_dev is NULL");
    for (int i = 0; i < n_m; ++i)
        if (!D_dev[i]) return fail(PASTILA_EINVAL, "D_dev[%d] is NULL", i);
    TRY(set_device(h));
    std::vector<MParams> qs(n_m);
    for (int i = 0; i < n_m; ++i) TRY(resolve(h, m_list[i], rule, &qs[i]));
    if (h->prec == PASTILA_FP32) return profiles_batch_t<float, V_F32>(h, qs, D_dev, D_max_dev);
    // FP64: the plain path, one length after the other
    void* dk;
    TRY(scratch(h, "dmax", 8, &dk));
    for (int i = 0; i < n_m; ++i) {
        TRY(launch_profiles(h, qs[i], D_dev[i], (unsigned long long*)dk));
        if (D_max_dev) {
            dec_dmax_kernel<<<1, 1, 0, h->stream>>>((const unsigned long long*)dk, D_max_dev + i);
            CK(cudaGetLastError());
            h->launches += 1;
        }
    }
    return PASTILA_OK;
}

pastila_status pastila_set_fp64_ties(pastila_series* h, int on) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    h->fp64_ties = on != 0;
    auto& gr = h->graph;  // a captured sweep holds the previous choice
    for (auto& e : gr.exec)
        if (e) cudaGraphExecDestroy(e);
    gr.exec[0] = gr.exec[1] = gr.exec[2] = nullptr;
    gr.ms.clear();
    return PASTILA_OK;
}

pastila_status pastila_stage_status(pastila_series* h) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    return stage_check(h);
}

pastila_status pastila_profiles(pastila_series* h, int32_t m, pastila_mparams mp, void* D_out,
                                double* D_max_out) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    TRY(set_device(h));
    MParams q;
    TRY(resolve(h, m, mp, &q));
    const size_t bytes = real_size(h) * (size_t)q.S * (size_t)q.P;
    void *D, *dk;
    TRY(scratch(h, "D", bytes, &D));
    TRY(scratch(h, "dmax", 8, &dk));
    TRY(launch_profiles(h, q, D, (unsigned long long*)dk));
    if (D_out) CK(cudaMemcpyAsync(D_out, D, bytes, cudaMemcpyDeviceToHost, h->stream));
    unsigned long long key = 0;
    CK(cudaMemcpyAsync(&key, dk, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (D_max_out) *D_max_out = KeyOf<double>::dec(key);
    return stage_check(h);
}

pastila_status pastila_snippets(pastila_series* h, int32_t m, pastila_mparams mp, int32_t K,
                                pastila_snippet* out, int32_t* labels_out, void* snippet_profiles_out) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    if (!out) return fail(PASTILA_EINVAL, "out is NULL");
    TRY(set_device(h));
    MParams q;
    TRY(resolve(h, m, mp, &q));
    if (K < 1 || K > q.S || K > 64)
        return fail(PASTILA_EINVAL, "K = %d: must satisfy 1 <= K <= min(n / m, 64) = %d", K, q.S < 64 ? q.S : 64);
    const size_t rs = real_size(h);
    const size_t bytes = rs * (size_t)q.S * (size_t)q.P;
    void *D, *dk, *lab = nullptr;
    {
        const pastila_status sd = scratch(h, "D", bytes, &D);
        if (sd == PASTILA_ENOMEM) {  // D does not fit: search without it, same results
            g_err.clear();
            TRY(streamed(h, q, K, labels_out, snippet_profiles_out, nullptr));
            TRY(read_snippets(h, K, out));
            return stage_check(h);
        }
        TRY(sd);
    }
    TRY(scratch(h, "dmax", 8, &dk));
    if (labels_out) TRY(scratch(h, "labels", 4 * (size_t)q.P, &lab));
    TRY(launch_profiles(h, q, D, (unsigned long long*)dk));
    TRY(snippets_on_device(h, q, D, K, (int32_t*)lab, (const unsigned long long*)dk, nullptr));
    if (labels_out) CK(cudaMemcpyAsync(labels_out, lab, 4 * (size_t)q.P, cudaMemcpyDeviceToHost, h->stream));
    if (snippet_profiles_out) {
        std::vector<int32_t> chosen(K);
        CK(cudaMemcpyAsync(chosen.data(), h->bufs["sn_chosen"].p, 4 * K, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int t = 0; t < K; ++t)
            CK(cudaMemcpyAsync((char*)snippet_profiles_out + rs * (size_t)t * q.P,
                               (const char*)D + rs * (size_t)chosen[t] * q.P, rs * (size_t)q.P,
                               cudaMemcpyDeviceToHost, h->stream));
    }
    TRY(read_snippets(h, K, out));
    return stage_check(h);
}

pastila_status pastila_snippets_streamed(pastila_series* h, int32_t m, pastila_mparams mp, int32_t K,
                                         pastila_snippet* out, int32_t* labels_out, void* snippet_profiles_out,
                                         int64_t* work_out) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    if (!out) return fail(PASTILA_EINVAL, "out is NULL");
    TRY(set_device(h));
    MParams q;
    TRY(resolve(h, m, mp, &q));
    if (K < 1 || K > q.S || K > 64)
        return fail(PASTILA_EINVAL, "K = %d: must satisfy 1 <= K <= min(n / m, 64) = %d", K, q.S < 64 ? q.S : 64);
    TRY(streamed(h, q, K, labels_out, snippet_profiles_out, work_out));
    TRY(read_snippets(h, K, out));
    return stage_check(h);
}

pastila_status pastila_select_length(pastila_series* h, const int32_t* m_list, int32_t n_m, pastila_mparams rule,
                                     int32_t K, int32_t* m_best, double* crit_out, pastila_snippet* best_out) {
    g_err.clear();
    if (!h) return fail(PASTILA_EINVAL, "handle is NULL");
    if (!m_list || n_m < 1) return fail(PASTILA_EINVAL, "m_list is empty");
    if (!m_best) return fail(PASTILA_EINVAL, "m_best is NULL");
    TRY(set_device(h));
    std::vector<MParams> qs(n_m);
    int min_S = 1 << 30;
    for (int i = 0; i < n_m; ++i) {
        TRY(resolve(h, m_list[i], rule, &qs[i]));
        min_S = qs[i].S < min_S ? qs[i].S : min_S;
    }
    if (K < 2 || K > min_S || K > 64)
        return fail(PASTILA_EINVAL, "K = %d: must satisfy 2 <= K <= min(n / max m, 64) = %d", K,
                    min_S < 64 ? min_S : 64);
    if (h->prec == PASTILA_FP32) {
        TRY(select_length_batched_t<float, V_F32>(h, m_list, n_m, rule, qs, K, m_best, crit_out, best_out));
        return stage_check(h);
    }
    // FP64: the plain path, one length after the other
    const size_t rs = real_size(h);
    void *crit, *ms, *bi, *dk;
    TRY(scratch(h, "sel_crit", 8 * (size_t)n_m, &crit));
    TRY(scratch(h, "sel_ms", 4 * (size_t)n_m, &ms));
    TRY(scratch(h, "sel_best", 4, &bi));
    TRY(scratch(h, "dmax", 8, &dk));
    CK(cudaMemcpyAsync(ms, m_list, 4 * (size_t)n_m, cudaMemcpyHostToDevice, h->stream));
    std::vector<pastila_snippet> per_m((size_t)n_m * K);
    for (int i = 0; i < n_m; ++i) {
        const MParams& q = qs[i];
        void* D;
        TRY(scratch(h, "D", rs * (size_t)q.S * (size_t)q.P, &D));
        TRY(launch_profiles(h, q, D, (unsigned long long*)dk));
        TRY(snippets_on_device(h, q, D, K, nullptr, (const unsigned long long*)dk, (double*)crit + i));
        TRY(read_snippets(h, K, per_m.data() + (size_t)i * K));
    }
    select_best_kernel<<<1, 1, 0, h->stream>>>((const double*)crit, (const int32_t*)ms, n_m, (int32_t*)bi);
    CK(cudaGetLastError());
    h->launches += 1;
    int32_t b = 0;
    std::vector<double> cv(n_m);
    CK(cudaMemcpyAsync(&b, bi, 4, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(cv.data(), crit, 8 * (size_t)n_m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *m_best = m_list[b];
    if (crit_out) memcpy(crit_out, cv.data(), 8 * (size_t)n_m);
    if (best_out) memcpy(best_out, per_m.data() + (size_t)b * K, sizeof(pastila_snippet) * K);
    return stage_check(h);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free greedy snippet search.
//
// Some callers cannot call cudaMalloc: code running where device memory is
// owned by another allocator (a framework's caching pool, a memory-capped or
// pre-partitioned process) or where allocation is not allowed once the hot loop
// has started.  For them, pastila_greedy_noalloc runs the greedy search of
// eqs. 16-17 on a profile set they already hold in device memory, with its
// working storage (the per-segment areas and the representativeness curve M)
// in the fixed device array below instead of in allocated buffers.
//
// The array is defined once for the whole library and every GPU that loads
// the library holds it until the process exits.  Host code may not use its
// name as a device address: the address is looked up once per device with
// cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------
namespace {
constexpr int NOALLOC_MAX_S = 16384;              // segments
constexpr int64_t NOALLOC_MAX_P = 1 << 20;        // positions
constexpr size_t NOALLOC_AREA_BYTES = 8 * (size_t)NOALLOC_MAX_S;
constexpr size_t NOALLOC_BYTES = NOALLOC_AREA_BYTES + 4 * (size_t)NOALLOC_MAX_P;  // 4.125 MiB
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 128;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device; looked up on the
// first call made with that device current.
pastila_status noalloc_scratch(void** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return fail(PASTILA_EINVAL, "device %d: the allocation-free entry point supports devices 0..%d", dev,
                    NOALLOC_MAX_DEVICES - 1);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return PASTILA_OK;
}
}  // namespace

extern "C" pastila_status pastila_greedy_noalloc(const float* D_dev, int32_t S, int64_t P, int32_t K,
                                                 int32_t* chosen_dev, double* area_after_dev, void* stream) {
    g_err.clear();
    if (!D_dev || !chosen_dev || !area_after_dev)
        return fail(PASTILA_EINVAL, "D_dev, chosen_dev and area_after_dev must be device pointers");
    if (S < 1 || P < 1) return fail(PASTILA_EINVAL, "S = %d, P = %lld: both must be positive", S, (long long)P);
    if (S > NOALLOC_MAX_S)
        return fail(PASTILA_EINVAL, "S = %d exceeds the %d segments the fixed scratch holds", S, NOALLOC_MAX_S);
    if (P > NOALLOC_MAX_P)
        return fail(PASTILA_EINVAL, "P = %lld exceeds the %lld positions the fixed scratch holds", (long long)P,
                    (long long)NOALLOC_MAX_P);
    if (K < 1 || K > S || K > 64)
        return fail(PASTILA_EINVAL, "K = %d: must satisfy 1 <= K <= min(S, 64) = %d", K, S < 64 ? S : 64);
    void* base = nullptr;
    TRY(noalloc_scratch(&base));
    double* area = (double*)base;
    float* M = (float*)((unsigned char*)base + NOALLOC_AREA_BYTES);
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned pb = (unsigned)((P + 255) / 256);
    // every step writes all S areas and step 0 writes all of M before it is
    // read, so nothing left in the array by an earlier call is ever used
    for (int t = 0; t < K; ++t) {
        area_kernel<float><<<S, AREA_THREADS, 0, st>>>(D_dev, S, P, t ? M : nullptr, chosen_dev, t, area);
        argmin_area_kernel<<<1, 1024, 0, st>>>(area, S, chosen_dev, area_after_dev, t);
        if (t + 1 < K) update_curve_kernel<float><<<pb, 256, 0, st>>>(D_dev, P, chosen_dev, t, M);
    }
    CK(cudaGetLastError());
    return PASTILA_OK;
}

// ---------------------------------------------------------------------------
// Measured FMA rates (the roofline denominators of an ALU-bound kernel).
// ---------------------------------------------------------------------------
namespace {
template <typename T>
pastila_status fma_rate(int sms, int iters, double* tflops) {
    const int blocks = sms * 8, threads = 256;  // 8 CTAs of 256 threads per SM
    T* out = nullptr;
    CK(cudaMalloc((void**)&out, sizeof(T) * (size_t)blocks * threads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_probe_kernel<T><<<blocks, threads>>>(out, 8, (T)1);  // warm-up
    cudaEventRecord(e0);
    fma_probe_kernel<T><<<blocks, threads>>>(out, iters, (T)1);
    cudaEventRecord(e1);
    cudaError_t r = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (r != cudaSuccess) return fail(PASTILA_ECUDA, "fma probe: %s", cudaGetErrorString(r));
    const double fmas = (double)blocks * threads * iters * 16.0 * PROBE_CHAINS;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    return PASTILA_OK;
}
}  // namespace

extern "C" pastila_status pastila_probe_fma(int32_t device, double* fp32_tflops, double* fp64_tflops) {
    g_err.clear();
    if (!fp32_tflops || !fp64_tflops) return fail(PASTILA_EINVAL, "output pointers must not be NULL");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(PASTILA_EINVAL, "device %d: %d device(s) visible", device, ndev);
    CK(cudaSetDevice(device));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    TRY(fma_rate<float>(sms, 4096, fp32_tflops));
    TRY(fma_rate<double>(sms, 64, fp64_tflops));
    return PASTILA_OK;
}
