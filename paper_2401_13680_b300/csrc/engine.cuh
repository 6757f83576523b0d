// Serving engine: continuous batching of snippet jobs on one GPU.
//
// Included by pastila_api.cu after its helpers, so that the library is one
// translation unit and every kernel template has a single instantiation.
//
// A job is one series with its own length sweep (m_list, rule, K): the work of
// one select_length call (Section 4.1 profiles, eqs. 16-17 greedy search, eq. 18
// criterion, eqs. 6-8 records of m_best).  Its lengths are items.
//
//   admission  queued jobs leave the queue in arrival order while a slot is free
//              and their resident memory plus their largest profile set fits
//              the budget; a job that could never fit is refused when it is
//              submitted (ENOMEM)
//   resident   per admitted job, from admission to its last wave: the series,
//              the window statistics of each distinct ell, the K chosen
//              profiles of every length, the greedy/criterion state
//   items      the S x P profile set D of one (job, m) exists from the wave of
//              its first tile chunk until its greedy search has run
//   waves      one wave is one sequence of launches on the compute stream:
//                statistics of the jobs admitted in this wave,
//                ONE tile launch over segment ranges (chunks) of items of every
//                  active job -- the ED cells of a wave are shared equally among
//                  the active jobs, so a short job arriving behind a long one is
//                  not served after it (processor sharing),
//                the batched greedy search and criterion of every item whose
//                  tiles are all issued, then its K chosen rows are kept and D
//                  is freed,
//                m_best and the records of every job whose items are all done,
//                  and one copy of its results to pinned host memory
//   overlap    up to max_waves_in_flight waves are on the stream at once, so the
//              next wave (with the jobs that arrived meanwhile) is queued before
//              the running one ends; series uploads run on a separate copy
//              stream.
// Every tile, greedy and criterion value is computed by the kernels the
// select_length path uses, on the same tile geometry, so a job's results do not
// depend on what else shares its waves.
#pragma once
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>

#include "runtime_model.cuh"

namespace pastila {

template <typename real>
struct JobFinal {
    int n_m, K;
    const int32_t* ms;          // n_m lengths, in sweep order
    const int64_t* P;           // n_m position counts
    const int64_t* keep_off;    // n_m offsets (elements) of each length's K kept rows
    const real* keep;           // kept rows: row t of length u at keep + keep_off[u] + t * P[u]
    const int32_t* chosen;      // n_m x K chosen segments, greedy order
    const double* area_after;   // n_m x K
    const double* crit;         // n_m eq. 18 values
    int32_t* best;              // index of m_best in the sweep
    unsigned long long* counts; // K nearest-snippet counts of m_best
    int32_t* rec_index;
    int32_t* rec_rank;
    double* rec_frac;
    double* rec_area;
};

__global__ void engine_init_keys_kernel(unsigned long long* __restrict__ keys, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = KeyOf<double>::enc(0.0);
}

// keep[y][t * P + p] = D_{chosen[t]}(p) for the items of a greedy batch:
// grid (ceil(max P / 256), n items)
template <typename real>
__global__ void gather_chosen_kernel(const BatchItem<real>* __restrict__ items, real* const* __restrict__ keep) {
    const BatchItem<real>& it = items[blockIdx.y];
    const int64_t P = it.A.P;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    real* out = keep[blockIdx.y];
    for (int t = 0; t < it.K; ++t) out[(int64_t)t * P + p] = it.A.D[(int64_t)it.chosen[t] * P + p];
}

// m_best of each finishing job (largest eq. 18 value, smallest m on ties);
// clears its counts.  One CTA.
template <typename real>
__global__ void job_best_kernel(const JobFinal<real>* __restrict__ f, int nf) {
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const JobFinal<real>& J = f[i];
        int b = 0;
        for (int u = 1; u < J.n_m; ++u)
            if (J.crit[u] > J.crit[b] || (J.crit[u] == J.crit[b] && J.ms[u] < J.ms[b])) b = u;
        *J.best = b;
        for (int t = 0; t < J.K; ++t) J.counts[t] = 0;
    }
}

// eq. 6: nearest chosen profile per position of m_best (ties: lowest segment),
// counted per snippet.  grid (ceil(max P / 256), n jobs)
template <typename real>
__global__ void job_neighbors_kernel(const JobFinal<real>* __restrict__ f) {
    __shared__ unsigned int local[64];
    const JobFinal<real>& J = f[blockIdx.y];
    if (threadIdx.x < 64) local[threadIdx.x] = 0;
    __syncthreads();
    const int b = *J.best;
    const int64_t P = J.P[b];
    const real* rows = J.keep + J.keep_off[b];
    const int32_t* chosen = J.chosen + (int64_t)b * J.K;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) {
        int bt = 0;
        real bv = rows[p];
        for (int t = 1; t < J.K; ++t) {
            const real v = rows[(int64_t)t * P + p];
            if (v < bv || (v == bv && chosen[t] < chosen[bt])) {
                bv = v;
                bt = t;
            }
        }
        atomicAdd(&local[bt], 1u);
    }
    __syncthreads();
    if ((int)threadIdx.x < J.K && local[threadIdx.x])
        atomicAdd(&J.counts[threadIdx.x], (unsigned long long)local[threadIdx.x]);
}

// eqs. 7-8 records of m_best: frac descending, segment ascending on ties.
// One thread per job.
template <typename real>
__global__ void job_records_kernel(const JobFinal<real>* __restrict__ f, int nf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const JobFinal<real>& J = f[i];
    const int b = *J.best, K = J.K;
    const int32_t* chosen = J.chosen + (int64_t)b * K;
    const double* aafter = J.area_after + (int64_t)b * K;
    int order[64];
    for (int t = 0; t < K; ++t) order[t] = t;
    for (int u = 1; u < K; ++u) {
        const int x = order[u];
        int v = u - 1;
        while (v >= 0) {
            const int y = order[v];
            const bool before = J.counts[x] > J.counts[y] || (J.counts[x] == J.counts[y] && chosen[x] < chosen[y]);
            if (!before) break;
            order[v + 1] = y;
            --v;
        }
        order[v + 1] = x;
    }
    for (int u = 0; u < K; ++u) {
        const int t = order[u];
        J.rec_index[u] = chosen[t];
        J.rec_rank[u] = t;
        J.rec_frac[u] = (double)J.counts[t] / (double)J.P[b];
        J.rec_area[u] = aafter[t];
    }
}

}  // namespace pastila

namespace {

constexpr int ENGINE_MAX_SWEEP = 64;
constexpr int ENGINE_MAX_K = 64;
constexpr size_t ENGINE_RESULT_SLOT = 4096;  // >= 8 + 8 * 64 + 24 * 64

struct EStats {
    int ell = 0;
    int64_t C = 0;
    double* mu = nullptr;
    void* a = nullptr;
    void* df = nullptr;
    void* dg = nullptr;
    void* muh = nullptr;  // mu as hi + lo pairs
    void* mul = nullptr;
    // FP64 terms of an FP32 engine's jobs (the greedy re-evaluation's FP64 rows)
    void* a64 = nullptr;
    void* df64 = nullptr;
    void* dg64 = nullptr;
    void* muh64 = nullptr;
    void* mul64 = nullptr;
};

struct EItem {
    MParams q{};
    TileGeom g{};
    int ntiles = 0;
    int stats = 0;        // index into the job's statistics
    int state = 0;        // 0 waiting, 1 tiles in progress, 2 tiles all issued, 3 greedy issued
    int next_seg = 0;
    double cells_per_seg = 0.0;  // ED cells (halo included) of one segment's tiles
    void* dblock = nullptr;      // D, M, area (and, in FP32 engines, the greedy re-evaluation's buffers)
    size_t dbytes = 0;
    TileGeom g64{};              // FP64 tile layout of the re-evaluation's rows (FP32 engines)
    float* kappa = nullptr;      // FP32 engines: the windows' conditioning ratios for this length's R
    void* refine = nullptr;      // refine_bytes of the re-evaluation, then its state words
    int32_t* rst = nullptr;
    void* D = nullptr;
    void* M = nullptr;
    double* area = nullptr;
    void* keep = nullptr;        // K kept rows, in the resident block
    int32_t* chosen = nullptr;
    double* area_after = nullptr;
    double* crit_part = nullptr;
    double* crit = nullptr;
    unsigned long long* dmax = nullptr;
};

struct EJob {
    int64_t id = 0;
    int state = PASTILA_JOB_QUEUED;
    pastila_status status = PASTILA_OK;
    std::string msg;
    int64_t n = 0;
    std::vector<double> T;  // host copy until the upload is staged
    std::vector<int32_t> ms;
    int K = 0;
    std::vector<EItem> items;
    std::vector<EStats> stats;
    int64_t Cmax = 0;
    size_t res_bytes = 0, max_dbytes = 0;
    void* res = nullptr;
    double* T_dev = nullptr;
    void* Th = nullptr;  // T as hi + lo pairs (written with every length's statistics)
    void* Tl = nullptr;
    void* Th64 = nullptr;  // T as FP64 pairs (value, 0), FP32 engines
    void* Tl64 = nullptr;
    double* inv = nullptr;
    int32_t* flat = nullptr;
    int32_t* ms_dev = nullptr;
    int64_t* P_dev = nullptr;
    int64_t* keep_off_dev = nullptr;
    void* keep_base = nullptr;
    unsigned long long* counts = nullptr;
    char* result_dev = nullptr;
    size_t result_bytes = 0;
    std::vector<char> meta_host;
    void* meta_dev = nullptr;
    cudaEvent_t ev_copy = nullptr;
    int slot = -1;
    bool cancel_req = false;
    bool finalizing = false;
    double t_submit = -1, t_admit = -1, t_done = -1;
    int64_t first_wave = -1, last_wave = -1;
    double ed_cells = 0.0, profile_cells = 0.0;
    double pred_ms = 0.0;  // the runtime model's device time for the whole job, at submission
    int32_t m_best = 0;
    std::vector<double> crit;
    std::vector<pastila_snippet> recs;
};

struct EWave {
    int64_t id = 0;
    int slot = 0;
    double feat[RM_NF] = {0, 0, 0, 0, 0};  // runtime-model features of the wave's work
    double pred = -1.0;                     // the model's prediction when the wave was formed
    bool trained = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> recycle;
    std::vector<int64_t> finals;
};

inline size_t up256e(size_t x) { return (x + 255) & ~(size_t)255; }

// Runtime-model features of a job's remaining work: the tile cells of the
// segments not yet issued and the greedy reads of the lengths whose search is
// not yet issued (the per-wave feature is left at 0).
template <typename real>
void job_features(const EJob& j, double* f) {
    for (int i = 0; i < RM_NF; ++i) f[i] = 0.0;
    for (const EItem& it : j.items) {
        if (it.state < 2) rm_add_cells(f, (double)(it.q.S - it.next_seg) * it.cells_per_seg, it.q.m);
        if (it.state < 3) f[3] += (double)j.K * (double)it.q.S * (double)it.q.P * (double)sizeof(real) * 1e-9;
    }
}

}  // namespace

struct pastila_engine {
    int device = 0;
    pastila_precision prec = PASTILA_FP32;
    size_t budget = 0, held = 0, peak = 0, reserve = 0;
    int max_active = 0, max_inflight = 0;
    double wave_cells = 0.0;
    double age_weight = 0.0;
    int policy = PASTILA_POLICY_SHARE;
    bool refine = true;  // FP32: near-tied greedy steps decided on FP64 areas
    FILE* job_log = nullptr;  // one JSON line per job that ends (pastila_engine_config.job_log_path)
    ~pastila_engine() {
        if (job_log) fclose(job_log);
    }
    int fail_at = 0;
    int* err = nullptr;  // host-mapped flag the tile kernels set when a bounded wait runs out
    long long spin_limit = 1ll << 31;
    int test_timeout = 0;
    pastila_status broken_status = PASTILA_ECUDA;
    int64_t alloc_count = 0;
    int smem_optin = 0;
    cudaStream_t cs = nullptr, xs = nullptr;
    cudaMemPool_t pool = nullptr;
    std::thread thr;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    bool stop = false;
    bool broken = false;
    std::string broken_msg;
    std::chrono::steady_clock::time_point t0;
    int64_t next_id = 1;
    int64_t next_wave = 0;
    std::map<int64_t, std::unique_ptr<EJob>> jobs;
    std::deque<int64_t> pending;
    std::vector<int64_t> active;  // admitted, not finalizing, in admission order
    int holding = 0;              // admitted and not yet harvested
    std::deque<EWave> inflight;
    std::vector<cudaEvent_t> ev_free;
    std::vector<int> slots_free;
    char* results_host = nullptr;  // pinned, max_active slots
    size_t desc_bytes = 0, cap_items = 0;
    std::vector<char*> desc_host;  // pinned, one per wave in flight
    std::vector<char*> desc_dev;
    // counters
    uint64_t n_submitted = 0, n_done = 0, n_failed = 0, n_cancelled = 0, n_waves = 0, launches = 0;
    double ed_cells = 0.0, profile_cells = 0.0, busy_ms = 0.0;
    uint64_t model_obs = 0, model_err_n = 0;
    double model_err_sum = 0.0;
};

namespace {

double eng_now(const pastila_engine* e) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - e->t0).count();
}

pastila_status eng_alloc(pastila_engine* e, void** p, size_t bytes, cudaStream_t s) {
    ++e->alloc_count;
    if (e->fail_at && e->alloc_count == e->fail_at)
        return fail(PASTILA_ENOMEM, "device allocation %lld failed (injected)", (long long)e->alloc_count);
    cudaError_t r = cudaMallocFromPoolAsync(p, bytes ? bytes : 256, e->pool, s);
    if (r == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(PASTILA_ENOMEM, "device allocation of %zu bytes failed: out of device memory", bytes);
    }
    if (r != cudaSuccess) return fail(PASTILA_ECUDA, "cudaMallocFromPoolAsync: %s", cudaGetErrorString(r));
    e->held += bytes;
    e->peak = std::max(e->peak, e->held);
    return PASTILA_OK;
}

void eng_free(pastila_engine* e, void*& p, size_t bytes) {
    if (!p) return;
    cudaFreeAsync(p, e->cs);  // stream-ordered after every launch that uses it
    e->held -= bytes;
    p = nullptr;
}

pastila_status eng_event(pastila_engine* e, cudaEvent_t* ev) {
    if (!e->ev_free.empty()) {
        *ev = e->ev_free.back();
        e->ev_free.pop_back();
        return PASTILA_OK;
    }
    CK(cudaEventCreate(ev));
    return PASTILA_OK;
}

// The job's JSON line in the engine's log (messages keep printable ASCII only,
// quotes and backslashes escaped).
void log_job(pastila_engine* e, const EJob& j) {
    if (!e->job_log) return;
    static const char* const names[5] = {"queued", "active", "done", "failed", "cancelled"};
    std::string msg;
    for (char ch : j.msg) {
        if (ch == '"' || ch == '\\') msg += '\\';
        if (ch >= 32 && ch < 127) msg += ch;
    }
    std::string ms;
    for (size_t i = 0; i < j.ms.size(); ++i) ms += (i ? ", " : "") + std::to_string(j.ms[i]);
    fprintf(e->job_log,
            "{\"job\": %lld, \"state\": \"%s\", \"status\": %d, \"message\": \"%s\", \"n\": %lld, "
            "\"m_list\": [%s], \"K\": %d, \"t_submit\": %.6f, \"t_admit\": %.6f, \"t_done\": %.6f, "
            "\"latency_s\": %.6f, \"first_wave\": %lld, \"last_wave\": %lld, \"ed_cells\": %.6g, "
            "\"profile_cells\": %.6g, \"mem_bytes\": %zu, \"predicted_ms\": %.3f, \"m_best\": %d}\n",
            (long long)j.id, names[j.state < 0 || j.state > 4 ? 0 : j.state], (int)j.status, msg.c_str(),
            (long long)j.n, ms.c_str(), j.K, j.t_submit, j.t_admit, j.t_done, j.t_done - j.t_submit,
            (long long)j.first_wave, (long long)j.last_wave, j.ed_cells, j.profile_cells,
            j.res_bytes + j.max_dbytes, j.pred_ms, j.state == PASTILA_JOB_DONE ? (int)j.m_best : 0);
    fflush(e->job_log);
}

void job_final_state(pastila_engine* e, EJob& j, int state, pastila_status st, const std::string& msg) {
    j.state = state;
    j.status = st;
    j.msg = msg;
    j.t_done = eng_now(e);
    if (state == PASTILA_JOB_DONE) e->n_done++;
    if (state == PASTILA_JOB_FAILED) e->n_failed++;
    if (state == PASTILA_JOB_CANCELLED) e->n_cancelled++;
    log_job(e, j);
    j.T.clear();
    j.T.shrink_to_fit();
    e->cv_done.notify_all();
}

// Sizes, tile geometry and memory of a job, from its arguments alone.
template <typename real, int V>
pastila_status plan_job(pastila_engine* e, EJob& j, pastila_mparams rule) {
    const size_t rs = sizeof(real);
    const int n_m = (int)j.ms.size();
    j.items.assign(n_m, EItem{});
    int min_S = 1 << 30;
    for (int u = 0; u < n_m; ++u) {
        EItem& it = j.items[u];
        TRY(resolve_n(j.n, j.ms[u], rule, &it.q));
        TRY(choose_tile_s<real, V>((size_t)e->smem_optin, it.q, &it.g));
        it.ntiles = (int)((it.q.P + it.g.W - 1) / it.g.W);
        it.cells_per_seg = (double)it.ntiles * (double)it.q.R * (double)it.g.Wb;
        min_S = std::min(min_S, it.q.S);
        int si = -1;
        for (int w = 0; w < (int)j.stats.size(); ++w)
            if (j.stats[w].ell == it.q.ell) si = w;
        if (si < 0) {
            EStats st;
            st.ell = it.q.ell;
            st.C = it.q.C;
            j.stats.push_back(st);
            si = (int)j.stats.size() - 1;
        }
        it.stats = si;
        it.dbytes = up256e(rs * (size_t)it.q.S * (size_t)it.q.P) + up256e(rs * (size_t)it.q.P) +
                    up256e(8 * (size_t)it.q.S);
        if (std::is_same<real, float>::value && e->refine) {  // the greedy re-evaluation's FP64 rows and state
            TRY(choose_tile_s<double, V_F64>((size_t)e->smem_optin, it.q, &it.g64));
            it.dbytes += refine_bytes(it.q, j.K) + up256e(4 * REF_STATE_INTS);
        }
        j.max_dbytes = std::max(j.max_dbytes, it.dbytes);
        j.ed_cells += it.cells_per_seg * it.q.S;
        j.profile_cells += (double)it.q.S * (double)it.q.P;
    }
    const int K = j.K;
    if (K < 2 || K > min_S || K > ENGINE_MAX_K)
        return fail(PASTILA_EINVAL, "K = %d: must satisfy 2 <= K <= min(n / max m, 64) = %d", K, std::min(min_S, 64));
    j.Cmax = 0;
    // the tile kernels' bulk copies may read up to 16 bytes past an array's end
    const bool refine = std::is_same<real, float>::value && e->refine;  // FP64 statistics for the greedy re-evaluation
    size_t b = up256e(8 * (size_t)j.n) + 2 * up256e(rs * (size_t)(j.n + ARRAY_PAD));
    if (refine) b += 2 * up256e(8 * (size_t)(j.n + ARRAY_PAD));
    for (auto& st : j.stats) {
        j.Cmax = std::max(j.Cmax, st.C);
        b += up256e(8 * (size_t)st.C) + 5 * up256e(rs * (size_t)(st.C + ARRAY_PAD));
        if (refine) b += 5 * up256e(8 * (size_t)(st.C + ARRAY_PAD));
    }
    b += up256e(8 * (size_t)j.Cmax) + up256e(4 * (size_t)j.Cmax);
    b += up256e(8 * (size_t)n_m) * 3;  // meta: ms (padded), P, keep_off
    for (auto& it : j.items) b += up256e(rs * (size_t)K * (size_t)it.q.P);
    if (std::is_same<real, float>::value)
        for (auto& it : j.items) b += up256e(4 * (size_t)(it.q.C + ARRAY_PAD));  // conditioning ratios
    b += up256e(4 * (size_t)n_m * K) + up256e(8 * (size_t)n_m * K) + up256e(8 * (size_t)n_m * CRIT_BLOCKS) +
         up256e(8 * (size_t)n_m) + up256e(8 * (size_t)K);
    j.result_bytes = 8 + 8 * (size_t)n_m + 24 * (size_t)K;
    b += up256e(j.result_bytes);
    j.res_bytes = b;
    return PASTILA_OK;
}

// Carves the resident block and stages the series and metadata on the copy stream.
template <typename real>
pastila_status admit_job(pastila_engine* e, EJob& j) {
    const size_t rs = sizeof(real);
    const int n_m = (int)j.ms.size(), K = j.K;
    char* p = (char*)j.res;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += up256e(bytes);
        return (void*)r;
    };
    const bool refine = std::is_same<real, float>::value && e->refine;
    j.T_dev = (double*)take(8 * (size_t)j.n);
    j.Th = take(rs * (size_t)(j.n + ARRAY_PAD));
    j.Tl = take(rs * (size_t)(j.n + ARRAY_PAD));
    if (refine) {
        j.Th64 = take(8 * (size_t)(j.n + ARRAY_PAD));
        j.Tl64 = take(8 * (size_t)(j.n + ARRAY_PAD));
    }
    for (auto& st : j.stats) {
        st.mu = (double*)take(8 * (size_t)st.C);
        st.a = take(rs * (size_t)(st.C + ARRAY_PAD));
        st.df = take(rs * (size_t)(st.C + ARRAY_PAD));
        st.dg = take(rs * (size_t)(st.C + ARRAY_PAD));
        st.muh = take(rs * (size_t)(st.C + ARRAY_PAD));
        st.mul = take(rs * (size_t)(st.C + ARRAY_PAD));
        if (refine) {
            st.a64 = take(8 * (size_t)(st.C + ARRAY_PAD));
            st.df64 = take(8 * (size_t)(st.C + ARRAY_PAD));
            st.dg64 = take(8 * (size_t)(st.C + ARRAY_PAD));
            st.muh64 = take(8 * (size_t)(st.C + ARRAY_PAD));
            st.mul64 = take(8 * (size_t)(st.C + ARRAY_PAD));
        }
    }
    j.inv = (double*)take(8 * (size_t)j.Cmax);
    j.flat = (int32_t*)take(4 * (size_t)j.Cmax);
    j.meta_dev = p;
    j.ms_dev = (int32_t*)take(8 * (size_t)n_m);
    j.P_dev = (int64_t*)take(8 * (size_t)n_m);
    j.keep_off_dev = (int64_t*)take(8 * (size_t)n_m);
    const size_t meta_bytes = (size_t)(p - (char*)j.meta_dev);
    j.keep_base = p;
    std::vector<int64_t> keep_off(n_m);
    for (int u = 0; u < n_m; ++u) {
        keep_off[u] = (int64_t)((p - (char*)j.keep_base) / rs);
        j.items[u].keep = take(rs * (size_t)K * (size_t)j.items[u].q.P);
    }
    if (std::is_same<real, float>::value)
        for (int u = 0; u < n_m; ++u) j.items[u].kappa = (float*)take(4 * (size_t)(j.items[u].q.C + ARRAY_PAD));
    int32_t* chosen = (int32_t*)take(4 * (size_t)n_m * K);
    double* aafter = (double*)take(8 * (size_t)n_m * K);
    double* cpart = (double*)take(8 * (size_t)n_m * CRIT_BLOCKS);
    unsigned long long* dmax = (unsigned long long*)take(8 * (size_t)n_m);
    j.counts = (unsigned long long*)take(8 * (size_t)K);
    j.result_dev = (char*)take(j.result_bytes);
    double* crit = (double*)(j.result_dev + 8);
    for (int u = 0; u < n_m; ++u) {
        EItem& it = j.items[u];
        it.chosen = chosen + (size_t)u * K;
        it.area_after = aafter + (size_t)u * K;
        it.crit_part = cpart + (size_t)u * CRIT_BLOCKS;
        it.crit = crit + u;
        it.dmax = dmax + u;
    }
    // metadata in the device layout: ms (int32, padded), P, keep_off
    j.meta_host.assign(meta_bytes, 0);
    char* mh = j.meta_host.data();
    for (int u = 0; u < n_m; ++u) {
        ((int32_t*)mh)[u] = j.ms[u];
        ((int64_t*)(mh + ((char*)j.P_dev - (char*)j.meta_dev)))[u] = j.items[u].q.P;
        ((int64_t*)(mh + ((char*)j.keep_off_dev - (char*)j.meta_dev)))[u] = keep_off[u];
    }
    // pageable copies on the copy stream return once the host data is staged
    CK(cudaMemcpyAsync(j.T_dev, j.T.data(), 8 * (size_t)j.n, cudaMemcpyHostToDevice, e->xs));
    CK(cudaMemcpyAsync(j.meta_dev, j.meta_host.data(), meta_bytes, cudaMemcpyHostToDevice, e->xs));
    TRY(eng_event(e, &j.ev_copy));
    CK(cudaEventRecord(j.ev_copy, e->xs));
    j.T.clear();
    j.T.shrink_to_fit();
    j.meta_host.clear();
    return PASTILA_OK;
}

template <typename real>
BatchItem<real> item_desc(const pastila_engine* e, const EJob& j, const EItem& it) {
    BatchItem<real> bi{};
    ProfileArgs<real>& A = bi.A;
    const EStats& st = j.stats[it.stats];
    A.Th = (const real*)j.Th;
    A.Tl = (const real*)j.Tl;
    A.muh = (const real*)st.muh;
    A.mul = (const real*)st.mul;
    A.a = (const real*)st.a;
    A.df = (const real*)st.df;
    A.dg = (const real*)st.dg;
    A.n = j.n;
    A.C = it.q.C;
    A.P = it.q.P;
    A.m = it.q.m;
    A.ell = it.q.ell;
    A.k = it.q.k;
    A.R = it.q.R;
    A.S = it.q.S;
    A.W = it.g.W;
    A.ntiles = it.ntiles;
    A.D = (real*)it.D;
    A.dmax_key = it.dmax;
    A.kappa = it.kappa;
    A.err = e->err;
    A.spin_limit = e->spin_limit;
    A.test_timeout = e->test_timeout;
    bi.G = it.g;
    bi.M = (real*)it.M;
    bi.area = it.area;
    bi.chosen = it.chosen;
    bi.area_after = it.area_after;
    bi.crit_part = it.crit_part;
    bi.crit = it.crit;
    bi.K = j.K;
    if (it.refine) {  // FP32 engine: the greedy re-evaluation's FP64 rows (cf. refine_attach)
        ProfileArgs<double> A64{};
        A64.Th = (const double*)j.Th64;
        A64.Tl = (const double*)j.Tl64;
        A64.muh = (const double*)st.muh64;
        A64.mul = (const double*)st.mul64;
        A64.a = (const double*)st.a64;
        A64.df = (const double*)st.df64;
        A64.dg = (const double*)st.dg64;
        A64.n = j.n;
        A64.C = it.q.C;
        A64.P = it.q.P;
        A64.m = it.q.m;
        A64.ell = it.q.ell;
        A64.k = it.q.k;
        A64.R = it.q.R;
        A64.S = it.q.S;
        A64.W = it.g64.W;
        A64.ntiles = (int)((it.q.P + it.g64.W - 1) / it.g64.W);
        A64.err = e->err;
        A64.spin_limit = e->spin_limit;
        A64.test_timeout = e->test_timeout;
        char* r = (char*)it.refine;
        bi.rows64 = (double*)r;
        r += up256e(8 * (size_t)(j.K + REF_NCAND) * (size_t)it.q.P);
        bi.bound = (float*)r;
        r += up256e(4 * (size_t)it.q.S);
        bi.cand_area = (double*)r;
        r += up256e(8 * REF_NCAND);
        A64.dmax_key = (unsigned long long*)r;
        r += up256e(8);
        bi.need = (uint8_t*)r;
        A64.D = bi.rows64;
        bi.A64 = A64;
        bi.G64 = it.g64;
        bi.rst = it.rst;
        bi.bc = (float)(2.2 * it.q.ell * REF_DRHO);
    }
    return bi;
}

void free_job_device(pastila_engine* e, EJob& j) {
    for (auto& it : j.items) eng_free(e, it.dblock, it.dbytes);
    eng_free(e, j.res, j.res_bytes);
}

struct Chunk {
    EJob* job;
    int item;
    int s0, segs;
};

// Plans and enqueues one wave; returns false when there is nothing to do.
template <typename real, int V>
pastila_status form_wave_t(pastila_engine* e, bool* did) {
    NvtxRange range("pastila: engine wave");
    *did = false;
    const int64_t wave_id = e->next_wave;
    std::vector<EJob*> admitted;
    std::vector<cudaEvent_t> recycle;
    bool changed = false;
    // 1. cancelled active jobs give back their memory and slot
    for (size_t a = 0; a < e->active.size();) {
        EJob& j = *e->jobs[e->active[a]];
        if (!j.cancel_req) {
            ++a;
            continue;
        }
        free_job_device(e, j);
        e->slots_free.push_back(j.slot);
        e->holding--;
        job_final_state(e, j, PASTILA_JOB_CANCELLED, PASTILA_ECANCELLED, "cancelled");
        e->active.erase(e->active.begin() + a);
        changed = true;
    }
    // 2. admission in arrival order, or (shortest-remaining-first policy) in
    // order of the jobs' predicted device time, arrival order among equals
    if (e->policy == PASTILA_POLICY_SRPT && e->pending.size() > 1)
        std::stable_sort(e->pending.begin(), e->pending.end(),
                         [e](int64_t x, int64_t y) { return e->jobs[x]->pred_ms < e->jobs[y]->pred_ms; });
    while (!e->pending.empty() && e->holding < e->max_active) {
        EJob& j = *e->jobs[e->pending.front()];
        if (j.cancel_req) {
            job_final_state(e, j, PASTILA_JOB_CANCELLED, PASTILA_ECANCELLED, "cancelled before admission");
            e->pending.pop_front();
            changed = true;
            continue;
        }
        if (e->held + e->reserve + j.res_bytes + j.max_dbytes > e->budget) break;  // wait for memory
        pastila_status st = eng_alloc(e, &j.res, j.res_bytes, e->xs);
        if (st != PASTILA_OK) {
            if (e->holding > 0 && st == PASTILA_ENOMEM && !(e->fail_at && e->alloc_count == e->fail_at))
                break;  // memory will come back when running jobs finish
            job_final_state(e, j, PASTILA_JOB_FAILED, st, g_err);
            e->pending.pop_front();
            changed = true;
            continue;
        }
        st = admit_job<real>(e, j);
        if (st != PASTILA_OK) return st;
        j.slot = e->slots_free.back();
        e->slots_free.pop_back();
        e->holding++;
        j.state = PASTILA_JOB_ACTIVE;
        j.t_admit = eng_now(e);
        e->pending.pop_front();
        e->active.push_back(j.id);
        admitted.push_back(&j);
        recycle.push_back(j.ev_copy);
        changed = true;
    }
    // 3. tile chunks: equal shares of the wave's ED cells, then the leftover in order
    std::vector<Chunk> chunks;
    std::vector<EJob*> with_work;
    for (int64_t id : e->active) {
        EJob& j = *e->jobs[id];
        for (auto& it : j.items)
            if (it.state < 2) {
                with_work.push_back(&j);
                break;
            }
    }
    size_t reserve = 0;
    double used = 0.0;
    auto take = [&](EJob& j, double quota) -> pastila_status {
        double taken = 0.0;
        for (int u = 0; u < (int)j.items.size() && taken < quota; ++u) {
            EItem& it = j.items[u];
            if (it.state >= 2) continue;
            if (it.state == 0) {
                if (e->held + reserve + it.dbytes > e->budget) {
                    reserve += it.dbytes;  // younger jobs leave this much for it
                    return PASTILA_OK;
                }
                pastila_status st = eng_alloc(e, &it.dblock, it.dbytes, e->cs);
                if (st == PASTILA_ENOMEM && !e->inflight.empty()) {
                    reserve += it.dbytes;
                    return PASTILA_OK;
                }
                if (st != PASTILA_OK) return st;
                char* p = (char*)it.dblock;
                it.D = p;
                p += up256e(sizeof(real) * (size_t)it.q.S * (size_t)it.q.P);
                it.M = p;
                p += up256e(sizeof(real) * (size_t)it.q.P);
                it.area = (double*)p;
                p += up256e(8 * (size_t)it.q.S);
                if (std::is_same<real, float>::value && e->refine) {
                    it.refine = p;
                    p += refine_bytes(it.q, j.K);
                    it.rst = (int32_t*)p;
                }
                it.state = 1;
                it.next_seg = 0;
            }
            const int avail = it.q.S - it.next_seg;
            const double fit = std::floor((quota - taken) / it.cells_per_seg);
            const int want = fit < 1.0 ? 1 : (fit >= (double)avail ? avail : (int)fit);
            if (!chunks.empty() && chunks.back().job == &j && chunks.back().item == u) {
                chunks.back().segs += want;
            } else {
                chunks.push_back(Chunk{&j, u, it.next_seg, want});
            }
            it.next_seg += want;
            taken += want * it.cells_per_seg;
            used += want * it.cells_per_seg;
            if (it.next_seg == it.q.S) it.state = 2;
        }
        return PASTILA_OK;
    };
    if (!with_work.empty() && e->policy == PASTILA_POLICY_SRPT) {
        // the whole wave to the job with the least predicted remaining device
        // time, then the next (admission order among equals)
        std::vector<double> rem(with_work.size());
        {
            std::lock_guard<std::mutex> lk(rm_table().mu);
            const RuntimeModel& rm = rm_table().m[e->prec == PASTILA_FP64];
            for (size_t i = 0; i < with_work.size(); ++i) {
                double f[RM_NF];
                job_features<real>(*with_work[i], f);
                rem[i] = rm.predict(f);
            }
        }
        std::vector<size_t> ord(with_work.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return rem[x] < rem[y]; });
        for (size_t i : ord)
            if (used < e->wave_cells) TRY(take(*with_work[i], e->wave_cells - used));
    } else if (!with_work.empty()) {
        // equal shares, or shares growing with the time since submission
        const double now = eng_now(e);
        std::vector<double> wt(with_work.size(), 1.0);
        double wsum = 0.0;
        for (size_t i = 0; i < with_work.size(); ++i) {
            if (e->age_weight > 0.0) wt[i] = 1.0 + (now - with_work[i]->t_submit) / e->age_weight;
            wsum += wt[i];
        }
        for (size_t i = 0; i < with_work.size(); ++i) TRY(take(*with_work[i], e->wave_cells * wt[i] / wsum));
        for (EJob* j : with_work)
            if (used < e->wave_cells) TRY(take(*j, e->wave_cells - used));
    }
    e->reserve = reserve;
    // chunks of one item must be contiguous in the list for the merge above;
    // the second pass may add a chunk of an item already in the list: merge those
    std::stable_sort(chunks.begin(), chunks.end(), [](const Chunk& x, const Chunk& y) {
        if (x.job->id != y.job->id) return x.job->id < y.job->id;
        if (x.item != y.item) return x.item < y.item;
        return x.s0 < y.s0;
    });
    std::vector<Chunk> merged;
    for (const Chunk& c : chunks) {
        if (!merged.empty() && merged.back().job == c.job && merged.back().item == c.item &&
            merged.back().s0 + merged.back().segs == c.s0)
            merged.back().segs += c.segs;
        else
            merged.push_back(c);
    }
    // 4. greedy batch: items whose tiles are all issued
    std::vector<std::pair<EJob*, int>> greedy;
    for (int64_t id : e->active) {
        EJob& j = *e->jobs[id];
        for (int u = 0; u < (int)j.items.size(); ++u)
            if (j.items[u].state == 2) greedy.push_back({&j, u});
    }
    // 5. jobs whose every item has its greedy search issued by the end of this wave
    std::vector<EJob*> finals;
    for (auto& gi : greedy) gi.first->items[gi.second].state = 3;
    for (size_t a = 0; a < e->active.size();) {
        EJob& j = *e->jobs[e->active[a]];
        bool all = true;
        for (auto& it : j.items) all &= it.state == 3;
        if (all) {
            finals.push_back(&j);
            j.finalizing = true;
            e->active.erase(e->active.begin() + a);
        } else {
            ++a;
        }
    }
    if (admitted.empty() && merged.empty() && greedy.empty() && finals.empty()) {
        *did = changed;
        return PASTILA_OK;
    }
    // descriptors into the pinned slot of this wave, then one upload
    const int slot = (int)(wave_id % e->max_inflight);
    char* hd = e->desc_host[slot];
    char* dd = e->desc_dev[slot];
    const size_t bi_bytes = up256e(sizeof(BatchItem<real>) * e->cap_items);
    const size_t kp_bytes = up256e(sizeof(real*) * e->cap_items);
    BatchItem<real>* h_tiles = (BatchItem<real>*)hd;
    BatchItem<real>* h_greedy = (BatchItem<real>*)(hd + bi_bytes);
    real** h_keep = (real**)(hd + 2 * bi_bytes);
    JobFinal<real>* h_fin = (JobFinal<real>*)(hd + 2 * bi_bytes + kp_bytes);
    double wave_cells = 0.0;
    double wfeat[RM_NF] = {0, 0, 0, 0, 1};
    // one tile launch per cluster size (a launch has a single cluster shape) and
    // apart the layouts that put two CTAs on an SM, each numbering its own CTAs
    const size_t lim = (size_t)e->smem_optin;
    auto cls = [lim](const TileGeom& g) { return 2 * g.CS + (pair_layout(g, lim) ? 1 : 0); };
    std::stable_sort(merged.begin(), merged.end(), [&](const Chunk& x, const Chunk& y) {
        return cls(x.job->items[x.item].g) < cls(y.job->items[y.item].g);
    });
    std::vector<TileGroup> groups;
    int gcls = -1;
    for (size_t c = 0; c < merged.size(); ++c) {
        const Chunk& ch = merged[c];
        const EItem& it = ch.job->items[ch.item];
        if (groups.empty() || gcls != cls(it.g)) {
            gcls = cls(it.g);
            TileGroup tg;
            tg.cs = it.g.CS;
            tg.first = (int)c;
            groups.push_back(tg);
        }
        TileGroup& tg = groups.back();
        h_tiles[c] = item_desc<real>(e, *ch.job, it);
        h_tiles[c].cta_begin = tg.ctas;
        h_tiles[c].s_begin = ch.s0;
        h_tiles[c].ctas = (long long)ch.segs * it.ntiles * it.g.CS;
        tg.ctas += h_tiles[c].ctas;
        tg.n++;
        tg.block = std::max(tg.block, it.g.NT);
        tg.smem = std::max(tg.smem, it.g.bytes);
        wave_cells += ch.segs * it.cells_per_seg;
        rm_add_cells(wfeat, ch.segs * it.cells_per_seg, it.q.m);
        if (ch.job->first_wave < 0) ch.job->first_wave = wave_id;
        ch.job->last_wave = wave_id;
    }
    int Kmax = 0;
    int64_t gmaxS = 0, gmaxP = 0;
    for (size_t g = 0; g < greedy.size(); ++g) {
        EJob& j = *greedy[g].first;
        const EItem& it = j.items[greedy[g].second];
        h_greedy[g] = item_desc<real>(e, j, it);
        h_keep[g] = (real*)it.keep;
        Kmax = std::max(Kmax, j.K);
        gmaxS = std::max<int64_t>(gmaxS, it.q.S);
        gmaxP = std::max<int64_t>(gmaxP, it.q.P);
        j.last_wave = wave_id;
    }
    for (size_t g = 0; g < greedy.size(); ++g) {  // every search runs Kmax area passes
        const EItem& it = greedy[g].first->items[greedy[g].second];
        wfeat[3] += (double)Kmax * (double)it.q.S * (double)it.q.P * (double)sizeof(real) * 1e-9;
    }
    int64_t fmaxP = 0;
    for (size_t f = 0; f < finals.size(); ++f) {
        EJob& j = *finals[f];
        JobFinal<real> F{};
        F.n_m = (int)j.ms.size();
        F.K = j.K;
        F.ms = j.ms_dev;
        F.P = j.P_dev;
        F.keep_off = j.keep_off_dev;
        F.keep = (const real*)j.keep_base;
        F.chosen = j.items[0].chosen;
        F.area_after = j.items[0].area_after;
        F.crit = (const double*)(j.result_dev + 8);
        F.best = (int32_t*)j.result_dev;
        F.counts = j.counts;
        const size_t n_m = j.ms.size();
        char* r = j.result_dev + 8 + 8 * n_m;
        F.rec_frac = (double*)r;
        F.rec_area = (double*)(r + 8 * (size_t)j.K);
        F.rec_index = (int32_t*)(r + 16 * (size_t)j.K);
        F.rec_rank = (int32_t*)(r + 20 * (size_t)j.K);
        h_fin[f] = F;
        for (auto& it : j.items) fmaxP = std::max<int64_t>(fmaxP, it.q.P);
        j.last_wave = wave_id;
    }
    const BatchItem<real>* d_tiles = (const BatchItem<real>*)dd;
    const BatchItem<real>* d_greedy = (const BatchItem<real>*)(dd + bi_bytes);
    real* const* d_keep = (real* const*)(dd + 2 * bi_bytes);
    const JobFinal<real>* d_fin = (const JobFinal<real>*)(dd + 2 * bi_bytes + kp_bytes);
    EWave w;
    w.id = wave_id;
    w.slot = slot;
    TRY(eng_event(e, &w.ev0));
    TRY(eng_event(e, &w.ev1));
    w.recycle = recycle;
    memcpy(w.feat, wfeat, sizeof wfeat);
    {
        std::lock_guard<std::mutex> lk(rm_table().mu);
        const RuntimeModel& rm = rm_table().m[e->prec == PASTILA_FP64];
        w.pred = rm.predict(wfeat);
        w.trained = rm.n >= RM_TRAINED;
    }
    cudaStream_t s = e->cs;
    CK(cudaEventRecord(w.ev0, s));
    if (!merged.empty())
        CK(cudaMemcpyAsync(dd, hd, sizeof(BatchItem<real>) * merged.size(), cudaMemcpyHostToDevice, s));
    if (!greedy.empty()) {
        CK(cudaMemcpyAsync(dd + bi_bytes, hd + bi_bytes, sizeof(BatchItem<real>) * greedy.size(),
                           cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dd + 2 * bi_bytes, hd + 2 * bi_bytes, sizeof(real*) * greedy.size(),
                           cudaMemcpyHostToDevice, s));
    }
    if (!finals.empty())
        CK(cudaMemcpyAsync(dd + 2 * bi_bytes + kp_bytes, hd + 2 * bi_bytes + kp_bytes,
                           sizeof(JobFinal<real>) * finals.size(), cudaMemcpyHostToDevice, s));
    uint64_t launches = 0;
    for (EJob* jp : admitted) {
        EJob& j = *jp;
        CK(cudaStreamWaitEvent(s, j.ev_copy, 0));
        for (auto& st : j.stats) {
            const int64_t nthr = (st.C + STATS_RUN - 1) / STATS_RUN;
            stats_mu_a_kernel<<<(unsigned)((nthr + 127) / 128), 128, 0, s>>>(j.T_dev, st.C, st.ell, st.mu, j.inv,
                                                                             j.flat);
            stats_terms_kernel<real><<<(unsigned)((j.n + 255) / 256), 256, 0, s>>>(
                j.T_dev, j.n, st.C, st.ell, st.mu, j.inv, (real*)st.a, (real*)st.df, (real*)st.dg,
                (real*)st.muh, (real*)st.mul, (real*)j.Th, (real*)j.Tl);
            launches += 2;
            if (st.a64) {  // FP64 terms for the greedy re-evaluation (same mu and inverse norms)
                stats_terms_kernel<double><<<(unsigned)((j.n + 255) / 256), 256, 0, s>>>(
                    j.T_dev, j.n, st.C, st.ell, st.mu, j.inv, (double*)st.a64, (double*)st.df64, (double*)st.dg64,
                    (double*)st.muh64, (double*)st.mul64, (double*)j.Th64, (double*)j.Tl64);
                launches += 1;
            }
        }
        for (auto& it : j.items) {  // FP32 tiles' conditioning ratios for each length's R
            if (!it.kappa) continue;
            const EStats& st = j.stats[it.stats];
            kappa_kernel<float><<<(unsigned)((it.q.C + 255) / 256), 256, 0, s>>>((const float*)st.a, it.q.C,
                                                                                it.q.R, it.kappa);
            launches += 1;
        }
        engine_init_keys_kernel<<<1, 64, 0, s>>>(j.items[0].dmax, (int)j.items.size());
        launches += 1;
    }
    for (const TileGroup& tg : groups) {
        CK(launch_tiles(batched_tiles_kernel<real, V>, dim3((unsigned)tg.ctas), tg.block, tg.smem, s, tg.cs,
                        d_tiles + tg.first, tg.n));
        launches += 1;
    }
    if (!greedy.empty()) {
        const int ng = (int)greedy.size();
        const unsigned pb = (unsigned)((gmaxP + 255) / 256);
        // the same greedy launches as select_length (with its FP64 re-evaluation of
        // near-tied steps on FP32 engines)
        const std::vector<BatchItem<real>> hg(h_greedy, h_greedy + ng);
        pastila_status gst;
        launches += (uint64_t)enqueue_greedy<real>(s, d_greedy, hg, Kmax, gmaxS, gmaxP, e->smem_optin, &gst);
        if (gst != PASTILA_OK) return gst;
        batched_criterion_kernel<real><<<dim3(CRIT_BLOCKS, ng), AREA_THREADS, 0, s>>>(d_greedy);
        batched_finish_kernel<real><<<1, 256, 0, s>>>(d_greedy, ng, nullptr);
        gather_chosen_kernel<real><<<dim3(pb, ng), 256, 0, s>>>(d_greedy, d_keep);
        launches += 3;
        for (auto& gi : greedy) {
            EItem& it = gi.first->items[gi.second];
            eng_free(e, it.dblock, it.dbytes);
        }
    }
    if (!finals.empty()) {
        const int nf = (int)finals.size();
        job_best_kernel<real><<<1, 64, 0, s>>>(d_fin, nf);
        job_neighbors_kernel<real><<<dim3((unsigned)((fmaxP + 255) / 256), nf), 256, 0, s>>>(d_fin);
        job_records_kernel<real><<<(nf + 63) / 64, 64, 0, s>>>(d_fin, nf);
        launches += 3;
        for (EJob* jp : finals) {
            CK(cudaMemcpyAsync(e->results_host + (size_t)jp->slot * ENGINE_RESULT_SLOT, jp->result_dev,
                               jp->result_bytes, cudaMemcpyDeviceToHost, s));
            eng_free(e, jp->res, jp->res_bytes);
            w.finals.push_back(jp->id);
        }
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(w.ev1, s));
    e->launches += launches;
    e->ed_cells += wave_cells;
    e->n_waves++;
    e->next_wave++;
    e->inflight.push_back(std::move(w));
    *did = true;
    return PASTILA_OK;
}

pastila_status form_wave(pastila_engine* e, bool* did) {
    if (e->prec == PASTILA_FP64) return form_wave_t<double, V_F64>(e, did);
    return form_wave_t<float, V_F32>(e, did);
}

void read_results(pastila_engine* e, EJob& j) {
    const char* r = e->results_host + (size_t)j.slot * ENGINE_RESULT_SLOT;
    const size_t n_m = j.ms.size();
    const int K = j.K;
    const int32_t b = *(const int32_t*)r;
    j.m_best = j.ms[b];
    j.crit.assign((const double*)(r + 8), (const double*)(r + 8) + n_m);
    const char* q = r + 8 + 8 * n_m;
    j.recs.resize(K);
    for (int u = 0; u < K; ++u) {
        j.recs[u].frac = ((const double*)q)[u];
        j.recs[u].area_after = ((const double*)(q + 8 * (size_t)K))[u];
        j.recs[u].index = ((const int32_t*)(q + 16 * (size_t)K))[u];
        j.recs[u].rank = ((const int32_t*)(q + 20 * (size_t)K))[u];
    }
}

void engine_break(pastila_engine* e, const std::string& msg) {
    e->broken = true;
    e->broken_msg = msg;
}

// Completed waves, oldest first.
void harvest(pastila_engine* e) {
    while (!e->inflight.empty()) {
        EWave& w = e->inflight.front();
        const cudaError_t q = cudaEventQuery(w.ev1);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) {
            cudaGetLastError();
            engine_break(e, std::string("wave failed: ") + cudaGetErrorString(q));
            return;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, w.ev0, w.ev1) == cudaSuccess) {
            e->busy_ms += ms;
            std::lock_guard<std::mutex> lk(rm_table().mu);
            rm_table().m[e->prec == PASTILA_FP64].observe(w.feat, (double)ms, w.pred, w.trained);
            e->model_obs++;
            if (w.trained && ms > 0.f) {
                e->model_err_sum += std::fabs(w.pred - (double)ms) / (double)ms;
                e->model_err_n++;
            }
        }
        if (*(volatile int*)e->err) {  // a tile of this wave (or an earlier one) gave up waiting
            e->broken_status = PASTILA_ETIMEOUT;
            engine_break(e, "a tile's staging copies did not complete within the wait limit");
            return;
        }
        for (int64_t id : w.finals) {
            EJob& j = *e->jobs[id];
            read_results(e, j);
            e->profile_cells += j.profile_cells;
            e->slots_free.push_back(j.slot);
            e->holding--;
            job_final_state(e, j, PASTILA_JOB_DONE, PASTILA_OK, "");
        }
        e->ev_free.push_back(w.ev0);
        e->ev_free.push_back(w.ev1);
        for (cudaEvent_t ev : w.recycle) e->ev_free.push_back(ev);
        e->inflight.pop_front();
        e->cv_done.notify_all();
    }
}

// Every job that is not finished ends with `st` (the engine is stopping or broken).
void end_all(pastila_engine* e, int state, pastila_status st, const std::string& msg) {
    for (auto& kv : e->jobs) {
        EJob& j = *kv.second;
        if (j.state == PASTILA_JOB_QUEUED || j.state == PASTILA_JOB_ACTIVE) {
            if (j.res || j.slot >= 0) free_job_device(e, j);
            job_final_state(e, j, state, st, msg);
        }
    }
    e->pending.clear();
    e->active.clear();
    e->cv_done.notify_all();
}

void scheduler(pastila_engine* e) {
    cudaSetDevice(e->device);
    std::unique_lock<std::mutex> lk(e->mu);
    while (true) {
        harvest(e);
        if (e->broken) {
            end_all(e, PASTILA_JOB_FAILED, e->broken_status, e->broken_msg);
            if (e->stop) break;
            e->cv_sched.wait(lk);
            continue;
        }
        if (e->stop) break;
        bool did = false;
        if ((int)e->inflight.size() < e->max_inflight) {
            pastila_status st = form_wave(e, &did);
            if (st != PASTILA_OK) {
                engine_break(e, g_err);
                continue;
            }
        }
        if (did) continue;
        if (!e->inflight.empty())
            e->cv_sched.wait_for(lk, std::chrono::microseconds(50));
        else
            e->cv_sched.wait(lk);
    }
    // stopping: the waves on the stream finish, queued and active jobs are cancelled
    lk.unlock();
    cudaStreamSynchronize(e->cs);
    lk.lock();
    harvest(e);
    end_all(e, PASTILA_JOB_CANCELLED, PASTILA_ECANCELLED, "engine destroyed");
    lk.unlock();
    cudaStreamSynchronize(e->cs);
}

pastila_status engine_job(pastila_engine* e, int64_t id, EJob** out) {
    auto it = e->jobs.find(id);
    if (it == e->jobs.end()) return fail(PASTILA_EINVAL, "job %lld is unknown (or released)", (long long)id);
    *out = it->second.get();
    return PASTILA_OK;
}

bool job_final(const EJob& j) {
    return j.state == PASTILA_JOB_DONE || j.state == PASTILA_JOB_FAILED || j.state == PASTILA_JOB_CANCELLED;
}

void engine_release_resources(pastila_engine* e) {
    for (char* p : e->desc_host)
        if (p) cudaFreeHost(p);
    for (char* p : e->desc_dev)
        if (p) cudaFree(p);
    if (e->results_host) cudaFreeHost(e->results_host);
    if (e->err) cudaFreeHost(e->err);
    for (cudaEvent_t ev : e->ev_free) cudaEventDestroy(ev);
    if (e->pool) cudaMemPoolDestroy(e->pool);
    if (e->cs) cudaStreamDestroy(e->cs);
    if (e->xs) cudaStreamDestroy(e->xs);
}

}  // namespace

extern "C" {

pastila_status pastila_engine_create(pastila_engine** out, const pastila_engine_config* cfg) {
    g_err.clear();
    if (!out) return fail(PASTILA_EINVAL, "out is NULL");
    *out = nullptr;
    pastila_engine_config c{};
    if (cfg) c = *cfg;
    if (c.prec != PASTILA_FP32 && c.prec != PASTILA_FP64) return fail(PASTILA_EINVAL, "unknown precision %d", (int)c.prec);
    if (c.max_active_jobs < 0 || c.max_active_jobs > 256)
        return fail(PASTILA_EINVAL, "max_active_jobs = %d: must be in [0, 256]", c.max_active_jobs);
    if (c.max_waves_in_flight < 0 || c.max_waves_in_flight > 8)
        return fail(PASTILA_EINVAL, "max_waves_in_flight = %d: must be in [0, 8]", c.max_waves_in_flight);
    if (!(c.wave_ed_cells >= 0.0)) return fail(PASTILA_EINVAL, "wave_ed_cells must be >= 0");
    if (c.fail_alloc_at < 0) return fail(PASTILA_EINVAL, "fail_alloc_at must be >= 0");
    if (!(c.age_weight_s >= 0.0)) return fail(PASTILA_EINVAL, "age_weight_s must be >= 0");
    if (c.policy != PASTILA_POLICY_SHARE && c.policy != PASTILA_POLICY_SRPT)
        return fail(PASTILA_EINVAL, "unknown policy %d", (int)c.policy);
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (c.device < 0 || c.device >= ndev) return fail(PASTILA_EINVAL, "device %d: %d device(s) visible", c.device, ndev);
    CK(cudaSetDevice(c.device));
    std::unique_ptr<pastila_engine> e(new pastila_engine());
    e->device = c.device;
    e->prec = c.prec;
    e->max_active = c.max_active_jobs ? c.max_active_jobs : 32;
    e->max_inflight = c.max_waves_in_flight ? c.max_waves_in_flight : 2;
    e->wave_cells = c.wave_ed_cells > 0.0 ? c.wave_ed_cells : 4e9;
    e->fail_at = c.fail_alloc_at;
    e->age_weight = c.age_weight_s;
    e->policy = c.policy;
    e->refine = c.prec == PASTILA_FP32 && c.fp32_greedy == 0;
    if (c.job_log_path && *c.job_log_path) {
        e->job_log = fopen(c.job_log_path, "a");
        if (!e->job_log) return fail(PASTILA_EINVAL, "cannot open the job log %s", c.job_log_path);
    }
    int smem = 0;
    CK(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device));
    e->smem_optin = smem - 1024;
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    e->budget = c.mem_budget_bytes ? c.mem_budget_bytes : (size_t)(0.9 * (double)fr);
    auto bail = [&](pastila_status s2) {
        engine_release_resources(e.get());
        return s2;
    };
    if (cudaStreamCreateWithFlags(&e->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&e->xs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(PASTILA_ECUDA, "cudaStreamCreate failed"));
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c.device;
    if (cudaMemPoolCreate(&e->pool, &props) != cudaSuccess) return bail(fail(PASTILA_ECUDA, "cudaMemPoolCreate failed"));
    uint64_t keep_all = ~0ull;  // keep freed memory in the pool
    cudaMemPoolSetAttribute(e->pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
    // an upload on the copy stream must never wait for the compute stream to reach
    // a free: reuse only memory whose free has already completed
    int no = 0;
    cudaMemPoolSetAttribute(e->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    e->cap_items = (size_t)e->max_active * ENGINE_MAX_SWEEP;
    const size_t bi = up256e(std::max(sizeof(BatchItem<float>), sizeof(BatchItem<double>)) * e->cap_items);
    const size_t kp = up256e(sizeof(void*) * e->cap_items);
    const size_t fin = up256e(std::max(sizeof(JobFinal<float>), sizeof(JobFinal<double>)) * (size_t)e->max_active);
    e->desc_bytes = 2 * bi + kp + fin;
    e->desc_host.assign(e->max_inflight, nullptr);
    e->desc_dev.assign(e->max_inflight, nullptr);
    for (int w = 0; w < e->max_inflight; ++w) {
        if (cudaMallocHost((void**)&e->desc_host[w], e->desc_bytes) != cudaSuccess ||
            cudaMalloc((void**)&e->desc_dev[w], e->desc_bytes) != cudaSuccess)
            return bail(fail(PASTILA_ENOMEM, "engine descriptor buffers (%zu bytes) could not be allocated",
                             e->desc_bytes));
    }
    if (cudaMallocHost((void**)&e->results_host, ENGINE_RESULT_SLOT * (size_t)e->max_active) != cudaSuccess)
        return bail(fail(PASTILA_ENOMEM, "engine result slots could not be allocated"));
    if (cudaHostAlloc((void**)&e->err, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
        return bail(fail(PASTILA_ENOMEM, "the engine's error flag could not be allocated"));
    *e->err = 0;
    wait_knobs(&e->spin_limit, &e->test_timeout);
    for (int q = e->max_active - 1; q >= 0; --q) e->slots_free.push_back(q);
    CK(tile_attrs(batched_tiles_kernel<float, V_F32>, e->smem_optin));
    CK(tile_attrs(batched_tiles_kernel<double, V_F64>, e->smem_optin));
    e->t0 = std::chrono::steady_clock::now();
    pastila_engine* ep = e.release();
    ep->thr = std::thread(scheduler, ep);
    *out = ep;
    return PASTILA_OK;
}

pastila_status pastila_engine_submit(pastila_engine* e, const double* T, int64_t n, const int32_t* m_list,
                                     int32_t n_m, pastila_mparams rule, int32_t K, int64_t* job_out) {
    g_err.clear();
    if (!e) return fail(PASTILA_EINVAL, "engine is NULL");
    if (!T) return fail(PASTILA_EINVAL, "T is NULL");
    if (!job_out) return fail(PASTILA_EINVAL, "job_out is NULL");
    if (n < 4) return fail(PASTILA_EINVAL, "n = %lld: the series needs at least 4 values", (long long)n);
    if (!m_list || n_m < 1 || n_m > ENGINE_MAX_SWEEP)
        return fail(PASTILA_EINVAL, "n_m = %d: a job sweeps 1 to %d lengths", n_m, ENGINE_MAX_SWEEP);
    TRY(check_finite(T, n));
    std::unique_ptr<EJob> j(new EJob());
    j->n = n;
    j->ms.assign(m_list, m_list + n_m);
    j->K = K;
    double f[RM_NF];
    if (e->prec == PASTILA_FP64) {
        TRY(plan_job<double, V_F64>(e, *j, rule));
        job_features<double>(*j, f);
    } else {
        TRY(plan_job<float, V_F32>(e, *j, rule));
        job_features<float>(*j, f);
    }
    f[4] = std::ceil(j->ed_cells / e->wave_cells);
    {
        std::lock_guard<std::mutex> lk(rm_table().mu);
        j->pred_ms = rm_table().m[e->prec == PASTILA_FP64].predict(f);
    }
    if (j->res_bytes + j->max_dbytes > e->budget)
        return fail(PASTILA_ENOMEM, "the job needs %zu bytes of device memory (resident %zu + largest profile set %zu); "
                    "the engine's budget is %zu", j->res_bytes + j->max_dbytes, j->res_bytes, j->max_dbytes, e->budget);
    j->T.assign(T, T + n);
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->broken) return fail(PASTILA_ECUDA, "the engine stopped after a device error: %s", e->broken_msg.c_str());
    if (e->stop) return fail(PASTILA_EINVAL, "the engine is shutting down");
    j->id = e->next_id++;
    j->t_submit = eng_now(e);
    *job_out = j->id;
    e->pending.push_back(j->id);
    e->jobs[j->id] = std::move(j);
    e->n_submitted++;
    e->cv_sched.notify_one();
    return PASTILA_OK;
}

pastila_status pastila_engine_submit_multi(pastila_engine* e, const double* T, int64_t n, int32_t d,
                                           const int32_t* m_list, int32_t n_m, pastila_mparams rule, int32_t K,
                                           int64_t* jobs_out) {
    g_err.clear();
    if (!e) return fail(PASTILA_EINVAL, "engine is NULL");
    if (!T) return fail(PASTILA_EINVAL, "T is NULL");
    if (!jobs_out) return fail(PASTILA_EINVAL, "jobs_out is NULL");
    if (d < 1 || d > 4096) return fail(PASTILA_EINVAL, "d = %d: 1 to 4096 coordinates", d);
    if (n < 4) return fail(PASTILA_EINVAL, "n = %lld: the series needs at least 4 values", (long long)n);
    if (!m_list || n_m < 1 || n_m > ENGINE_MAX_SWEEP)
        return fail(PASTILA_EINVAL, "n_m = %d: a job sweeps 1 to %d lengths", n_m, ENGINE_MAX_SWEEP);
    // every coordinate is checked and planned before any is queued
    std::vector<std::unique_ptr<EJob>> js;
    for (int c = 0; c < d; ++c) {
        const double* Tc = T + (size_t)c * (size_t)n;
        pastila_status st = check_finite(Tc, n);
        if (st != PASTILA_OK) return fail(st, "coordinate %d: %s", c, g_err.c_str());
        std::unique_ptr<EJob> j(new EJob());
        j->n = n;
        j->ms.assign(m_list, m_list + n_m);
        j->K = K;
        double f[RM_NF];
        if (e->prec == PASTILA_FP64) {
            TRY(plan_job<double, V_F64>(e, *j, rule));
            job_features<double>(*j, f);
        } else {
            TRY(plan_job<float, V_F32>(e, *j, rule));
            job_features<float>(*j, f);
        }
        f[4] = std::ceil(j->ed_cells / e->wave_cells);
        {
            std::lock_guard<std::mutex> lk(rm_table().mu);
            j->pred_ms = rm_table().m[e->prec == PASTILA_FP64].predict(f);
        }
        if (j->res_bytes + j->max_dbytes > e->budget)
            return fail(PASTILA_ENOMEM, "a coordinate needs %zu bytes of device memory; the engine's budget is %zu",
                        j->res_bytes + j->max_dbytes, e->budget);
        j->T.assign(Tc, Tc + n);
        js.push_back(std::move(j));
    }
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->broken) return fail(PASTILA_ECUDA, "the engine stopped after a device error: %s", e->broken_msg.c_str());
    if (e->stop) return fail(PASTILA_EINVAL, "the engine is shutting down");
    const double now = eng_now(e);
    for (int c = 0; c < d; ++c) {
        std::unique_ptr<EJob>& j = js[c];
        j->id = e->next_id++;
        j->t_submit = now;
        jobs_out[c] = j->id;
        e->pending.push_back(j->id);
        e->jobs[j->id] = std::move(j);
        e->n_submitted++;
    }
    e->cv_sched.notify_one();
    return PASTILA_OK;
}

pastila_status pastila_engine_poll(pastila_engine* e, int64_t job, int32_t timeout_ms, pastila_job_info* info) {
    g_err.clear();
    if (!e) return fail(PASTILA_EINVAL, "engine is NULL");
    std::unique_lock<std::mutex> lk(e->mu);
    EJob* j = nullptr;
    TRY(engine_job(e, job, &j));
    if (timeout_ms != 0 && !job_final(*j)) {
        auto pred = [&] { return job_final(*j); };
        if (timeout_ms < 0)
            e->cv_done.wait(lk, pred);
        else
            e->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    }
    if (info) {
        info->state = j->state;
        info->status = j->status;
        info->t_submit = j->t_submit;
        info->t_admit = j->t_admit;
        info->t_done = j->t_done;
        info->first_wave = j->first_wave;
        info->last_wave = j->last_wave;
        info->ed_cells = j->ed_cells;
        info->profile_cells = j->profile_cells;
        info->mem_bytes = j->res_bytes + j->max_dbytes;
        info->resident_bytes = j->res_bytes;
        info->predicted_ms = j->pred_ms;
    }
    if (!job_final(*j)) return fail(PASTILA_ETIMEOUT, "job %lld has not finished", (long long)job);
    return PASTILA_OK;
}

pastila_status pastila_engine_result(pastila_engine* e, int64_t job, int32_t* m_best, double* crit_out,
                                     pastila_snippet* best_out) {
    g_err.clear();
    if (!e) return fail(PASTILA_EINVAL, "engine is NULL");
    std::lock_guard<std::mutex> lk(e->mu);
    EJob* j = nullptr;
    TRY(engine_job(e, job, &j));
    if (!job_final(*j)) return fail(PASTILA_EBUSY, "job %lld has not finished", (long long)job);
    if (j->state == PASTILA_JOB_CANCELLED) return fail(PASTILA_ECANCELLED, "job %lld was cancelled", (long long)job);
    if (j->state == PASTILA_JOB_FAILED) return fail(j->status, "job %lld failed: %s", (long long)job, j->msg.c_str());
    if (m_best) *m_best = j->m_best;
    if (crit_out) memcpy(crit_out, j->crit.data(), 8 * j->crit.size());
    if (best_out) memcpy(best_out, j->recs.data(), sizeof(pastila_snippet) * j->recs.size());
    return PASTILA_OK;
}

pastila_status pastila_engine_cancel(pastila_engine* e, int64_t job) {
    g_err.clear();
    if (!e) return fail(PASTILA_EINVAL, "engine is NULL");
    std::lock_guard<std::mutex> lk(e->mu);
    EJob* j = nullptr;
    TRY(engine_job(e, job, &j));
    if (job_final(*j) || j->finalizing)
        return fail(PASTILA_EINVAL, "job %lld has finished or is finishing", (long long)job);
    j->cancel_req = true;
    e->cv_sched.notify_one();
    return PASTILA_OK;
}

pastila_status pastila_engine_release(pastila_engine* e, int64_t job) {
    g_err.clear();
    if (!e) return fail(PASTILA_EINVAL, "engine is NULL");
    std::lock_guard<std::mutex> lk(e->mu);
    EJob* j = nullptr;
    TRY(engine_job(e, job, &j));
    if (!job_final(*j)) return fail(PASTILA_EBUSY, "job %lld has not finished", (long long)job);
    e->jobs.erase(job);
    return PASTILA_OK;
}

pastila_status pastila_engine_stats(pastila_engine* e, pastila_engine_counters* out) {
    g_err.clear();
    if (!e || !out) return fail(PASTILA_EINVAL, "engine or out is NULL");
    std::lock_guard<std::mutex> lk(e->mu);
    out->submitted = e->n_submitted;
    out->done = e->n_done;
    out->failed = e->n_failed;
    out->cancelled = e->n_cancelled;
    out->waves = e->n_waves;
    out->launches = e->launches;
    out->ed_cells = e->ed_cells;
    out->profile_cells = e->profile_cells;
    out->busy_ms = e->busy_ms;
    out->mem_budget = e->budget;
    out->mem_held = e->held;
    out->mem_peak = e->peak;
    out->now = eng_now(e);
    out->model_waves = e->model_obs;
    out->model_rel_err = e->model_err_n ? e->model_err_sum / (double)e->model_err_n : -1.0;
    return PASTILA_OK;
}

void pastila_engine_destroy(pastila_engine* e) {
    if (!e) return;
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stop = true;
        e->cv_sched.notify_one();
    }
    if (e->thr.joinable()) e->thr.join();
    cudaSetDevice(e->device);
    engine_release_resources(e);
    delete e;
}

pastila_status pastila_model_get(pastila_precision prec, pastila_runtime_model* out) {
    g_err.clear();
    if (!out) return fail(PASTILA_EINVAL, "out is NULL");
    if (prec != PASTILA_FP32 && prec != PASTILA_FP64) return fail(PASTILA_EINVAL, "unknown precision %d", (int)prec);
    std::lock_guard<std::mutex> lk(rm_table().mu);
    const RuntimeModel& m = rm_table().m[prec == PASTILA_FP64];
    memset(out, 0, sizeof *out);
    out->prec = prec;
    out->n_coef = RM_NF;
    memcpy(out->coef, m.coef, sizeof m.coef);
    memcpy(out->prior, m.prior, sizeof m.prior);
    memcpy(out->xtx, m.xtx, sizeof m.xtx);
    memcpy(out->xty, m.xty, sizeof m.xty);
    out->observations = m.n;
    out->err_count = m.err_n;
    out->rel_err = m.err_n ? m.err_sum / (double)m.err_n : -1.0;
    return PASTILA_OK;
}

pastila_status pastila_model_set(const pastila_runtime_model* in) {
    g_err.clear();
    if (!in) return fail(PASTILA_EINVAL, "model is NULL");
    if (in->prec != PASTILA_FP32 && in->prec != PASTILA_FP64)
        return fail(PASTILA_EINVAL, "unknown precision %d", (int)in->prec);
    if (in->n_coef != RM_NF) return fail(PASTILA_EINVAL, "n_coef = %d: the model has %d coefficients", in->n_coef, RM_NF);
    for (int i = 0; i < RM_NF * RM_NF; ++i)
        if (!std::isfinite(in->xtx[i])) return fail(PASTILA_EINVAL, "xtx[%d] is not finite", i);
    for (int i = 0; i < RM_NF; ++i)
        if (!std::isfinite(in->xty[i]) || !std::isfinite(in->prior[i]))
            return fail(PASTILA_EINVAL, "xty[%d] or prior[%d] is not finite", i, i);
    std::lock_guard<std::mutex> lk(rm_table().mu);
    RuntimeModel& m = rm_table().m[in->prec == PASTILA_FP64];
    m.reset(in->prior);
    memcpy(m.xtx, in->xtx, sizeof m.xtx);
    memcpy(m.xty, in->xty, sizeof m.xty);
    m.n = in->observations;
    m.refit();
    return PASTILA_OK;
}

pastila_status pastila_model_observe(pastila_precision prec, const double* f, double ms) {
    g_err.clear();
    if (!f) return fail(PASTILA_EINVAL, "f is NULL");
    if (prec != PASTILA_FP32 && prec != PASTILA_FP64) return fail(PASTILA_EINVAL, "unknown precision %d", (int)prec);
    if (!(ms > 0.0) || !std::isfinite(ms)) return fail(PASTILA_EINVAL, "ms must be finite and > 0");
    for (int i = 0; i < RM_NF; ++i)
        if (!std::isfinite(f[i])) return fail(PASTILA_EINVAL, "f[%d] is not finite", i);
    std::lock_guard<std::mutex> lk(rm_table().mu);
    RuntimeModel& m = rm_table().m[prec == PASTILA_FP64];
    m.observe(f, ms, m.predict(f), m.n >= RM_TRAINED);
    return PASTILA_OK;
}

pastila_status pastila_model_reset(pastila_precision prec) {
    g_err.clear();
    if (prec != PASTILA_FP32 && prec != PASTILA_FP64) return fail(PASTILA_EINVAL, "unknown precision %d", (int)prec);
    std::lock_guard<std::mutex> lk(rm_table().mu);
    rm_table().m[prec == PASTILA_FP64].reset(rm_prior(prec == PASTILA_FP64));
    return PASTILA_OK;
}

pastila_status pastila_model_predict(pastila_precision prec, int64_t n, const int32_t* m_list, int32_t n_m,
                                     pastila_mparams rule, int32_t K, size_t smem_limit, double wave_ed_cells,
                                     double* ms_out) {
    g_err.clear();
    if (!ms_out) return fail(PASTILA_EINVAL, "ms_out is NULL");
    if (prec != PASTILA_FP32 && prec != PASTILA_FP64) return fail(PASTILA_EINVAL, "unknown precision %d", (int)prec);
    if (!m_list || n_m < 1 || n_m > ENGINE_MAX_SWEEP)
        return fail(PASTILA_EINVAL, "n_m = %d: a job sweeps 1 to %d lengths", n_m, ENGINE_MAX_SWEEP);
    if (!(wave_ed_cells >= 0.0)) return fail(PASTILA_EINVAL, "wave_ed_cells must be >= 0");
    const double rs = prec == PASTILA_FP64 ? 8.0 : 4.0;
    double f[RM_NF] = {0, 0, 0, 0, 0}, cells = 0.0;
    int min_S = 1 << 30;
    for (int u = 0; u < n_m; ++u) {
        MParams q;
        TRY(resolve_n(n, m_list[u], rule, &q));
        TileGeom g;
        if (prec == PASTILA_FP64)
            TRY(choose_tile_s<double, V_F64>(smem_limit, q, &g));
        else
            TRY(choose_tile_s<float, V_F32>(smem_limit, q, &g));
        const double ntiles = (double)((q.P + g.W - 1) / g.W);
        const double c = (double)q.S * ntiles * (double)q.R * (double)g.Wb;
        rm_add_cells(f, c, q.m);
        cells += c;
        f[3] += (double)K * (double)q.S * (double)q.P * rs * 1e-9;
        min_S = std::min(min_S, q.S);
    }
    if (K < 2 || K > min_S || K > ENGINE_MAX_K)
        return fail(PASTILA_EINVAL, "K = %d: must satisfy 2 <= K <= min(n / max m, 64) = %d", K, std::min(min_S, 64));
    f[4] = std::ceil(cells / (wave_ed_cells > 0.0 ? wave_ed_cells : 4e9));
    std::lock_guard<std::mutex> lk(rm_table().mu);
    *ms_out = rm_table().m[prec == PASTILA_FP64].predict(f);
    return PASTILA_OK;
}

}  // extern "C"
