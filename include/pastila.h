/*
 * pastila.h -- C ABI of the single-GPU MPdist-profile / snippet / length-selection
 * library (PaSTiLa, arXiv 2401.13680, Sections 3.2 and 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Indices are 0-based.  For a series T of n values and a snippet length m:
 *      segments   S_s = T[s*m .. s*m+m),  s = 0 .. S-1,  S = floor(n / m)   (eq. 4)
 *      positions  p = 0 .. P-1,  P = n - m + 1                            (eq. 14)
 *      ell        inner subsequence length, 2 <= ell <= m                 (eq. 9)
 *      R          = m - ell + 1 ell-subsequences per length-m window
 *      k          MPdist rank, k >= 1 (eq. 13)
 *  - D_s(p) = MPdist(S_s, T[p .. p+m)) (eqs. 14-15): the k-th smallest (1-based)
 *    of the 2R values of P_ABBA, or their largest when 2R <= k (eq. 13).
 *    P_ABBA joins, for the R x R block of z-normalised ell-subsequence distances
 *    between S_s and T[p .. p+m), its R row minima (eq. 11, window of R columns)
 *    and its R column minima (eq. 10).
 *  - Flat ell-windows (centred sum of squares <= 1e-24 * ell * max(1, mean^2)) have
 *    no z-normalisation: two flat windows are at distance 0, a flat and a
 *    non-flat window at sqrt(2 ell).  (The paper is silent; this is the library's
 *    reading.)
 *  - Every call returns a pastila_status and validates its arguments before any
 *    device work; on error nothing is written to the outputs and
 *    pastila_last_error() describes the failure.  No C++ exception crosses the ABI.
 *  - The library owns every handle and all device memory it allocates.  The
 *    caller owns every output buffer; "host" buffers are ordinary (pageable or
 *    pinned) host memory, "device" buffers are device pointers on the handle's
 *    device.  Calls on one handle are not thread-safe; separate handles are.
 *  - Results are deterministic: the same inputs give bit-identical outputs on
 *    the same device, alone or batched with other work.
 *  - Device-side waits are bounded.  The tile kernels wait once per tile, for
 *    the bulk copies that stage it; if that wait runs out (about a second) the
 *    tile raises a host-visible flag and still completes, and the next call
 *    on the handle that synchronises its stream (profiles, snippets,
 *    select_length, snippets_streamed, tune) returns PASTILA_ETIMEOUT with
 *    its outputs unspecified; an engine fails its unfinished jobs with
 *    PASTILA_ETIMEOUT and stops.  Callers of the enqueue-only entry points
 *    (pastila_profiles_device) read the flag with pastila_stage_status after
 *    synchronising.  The device context stays usable.  Before it ends, a tile
 *    whose wait ran out waits once more (bounded) for its copies, so that none
 *    lands after its shared memory is released; only if that second wait runs
 *    out as well can a copy still arrive late, into shared memory that another
 *    block of the same or a later kernel may own by then.
 *    (PASTILA_TEST_STAGE_WAIT=timeout in the environment when a handle or an
 *    engine is created makes every such wait run out, for tests.)
 */
#ifndef PASTILA_H_
#define PASTILA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pastila_series pastila_series; /* opaque: resident series + cached statistics */

typedef enum {
    PASTILA_OK = 0,
    PASTILA_EINVAL = 1,     /* an argument is out of range (message says which)          */
    PASTILA_ENOMEM = 2,     /* the work does not fit the memory budget or device memory  */
    PASTILA_ECUDA = 3,      /* a CUDA runtime call failed (message carries its string)   */
    PASTILA_ETIMEOUT = 4,   /* a bounded device-side wait ran out                        */
    PASTILA_ECANCELLED = 5, /* the job was cancelled before it finished                   */
    PASTILA_EBUSY = 6       /* the engine queue is full                                   */
} pastila_status;

typedef enum {
    PASTILA_FP32 = 0, /* FP32 covariance recurrence, exact FP32 seed per segment row 0 */
    PASTILA_FP64 = 1  /* the same algorithm in FP64 throughout (plain comparator path)  */
} pastila_precision;

/* MPdist parameters of one snippet length m.  ell = 0 selects m / 2 and k = 0
 * selects ceil(0.05 * 2m) = (m + 9) / 10, five per cent of 2m (Section 4.1). */
typedef struct {
    int32_t ell;
    int32_t k;
} pastila_mparams;

/* One snippet (eqs. 5-8): index is the segment number C.index; frac is the share
 * of positions whose nearest snippet it is (eq. 7); area_after is ProfileArea
 * (eq. 17) right after the greedy step that chose it; rank is that step (0-based). */
typedef struct {
    int32_t index;
    int32_t rank;
    double frac;
    double area_after;
} pastila_snippet;

/* ---------------------------------------------------------------- handle ---- */

/* Copies the n FP64 values of a host series T to device `device` and computes
 * nothing yet (window statistics are computed per ell on first use).
 * mem_budget_bytes bounds the device memory the handle may hold (0: no bound
 * beyond what the device has).  Errors: EINVAL (NULL out/T, n < 4, a non-finite
 * value, bad device or precision), ENOMEM, ECUDA. */
pastila_status pastila_create(pastila_series** out, const double* T, int64_t n, int device,
                              size_t mem_budget_bytes, pastila_precision prec);

/* As pastila_create, but T_dev is a device pointer (n FP64 values on `device`)
 * that the handle copies on `stream` (a cudaStream_t; NULL = a stream the handle
 * creates); the handle then issues all its work on that stream. */
pastila_status pastila_create_device(pastila_series** out, const double* T_dev, int64_t n,
                                     int device, size_t mem_budget_bytes,
                                     pastila_precision prec, void* stream);

/* Replaces the n resident values with new ones (same n) and marks every cached
 * ell-window statistic stale, so the next call recomputes it: for series that
 * are updated in place.  T: n host doubles; T_dev: n device doubles on the
 * handle's device, copied on the handle's stream.  Errors: EINVAL, ECUDA. */
pastila_status pastila_reload(pastila_series* h, const double* T);
pastila_status pastila_reload_device(pastila_series* h, const double* T_dev);

/* Frees the handle and every device buffer it owns (waits for its stream). */
void pastila_destroy(pastila_series* h);

/* Message of the last failed call on this thread ("" if none).  The pointer stays
 * valid until the next call on this thread. */
const char* pastila_last_error(void);

/* ----------------------------------------------------- profiles (eq. 15) ---- */

/* The profile set D = (D_0 .. D_{S-1}) for one m (eqs. 9-15) and its largest
 * value max_{s,p} D_s(p) (the denominator of eq. 18).
 * D_out: NULL, or a host buffer of S * P elements, row-major (segment-major),
 *        float for PASTILA_FP32 handles and double for PASTILA_FP64 handles.
 * D_max_out: NULL or one double.
 * Errors: EINVAL (m < 4 or m > n, ell or k out of range), ENOMEM, ECUDA. */
pastila_status pastila_profiles(pastila_series* h, int32_t m, pastila_mparams mp, void* D_out,
                                double* D_max_out);

/* As pastila_profiles with a device output buffer (same layout and element
 * type), written on the handle's stream; returns once the work is enqueued.
 * D_max_dev: NULL or a device double written on the same stream.
 * The call does not wait, so it cannot report a staging wait that ran out:
 * after synchronising the stream, call pastila_stage_status before using D. */
pastila_status pastila_profiles_device(pastila_series* h, int32_t m, pastila_mparams mp,
                                       void* D_dev, double* D_max_dev);

/* The profile sets of several lengths at once (eqs. 9-15 for each m of a
 * Section 4.2 length sweep), computed by the launch that pastila_select_length
 * makes for its sweep: on FP32 handles one batched tile launch per tile shape
 * covers every length; FP64 handles run the lengths one after another.
 * m_list: n_m lengths, each resolved with `rule` as pastila_select_length does
 *         (ell = 0: m/2; k = 0: ceil(m/10)).
 * D_dev:  n_m device pointers (a host array of them); D_dev[i] receives the
 *         S_i x P_i profile set of m_list[i], row-major, float (FP32 handles)
 *         or double (FP64 handles), S_i = floor(n / m_i), P_i = n - m_i + 1.
 * D_max_dev: NULL or n_m device doubles, the largest value of each set.
 * Every value equals the one pastila_profiles_device writes for that length
 * with the same tile layout, bit for bit.  Enqueued on the handle's stream,
 * like pastila_profiles_device (call pastila_stage_status after
 * synchronising).  Errors: EINVAL (empty list, a NULL buffer, m, ell or k out
 * of range), ENOMEM, ECUDA. */
pastila_status pastila_profiles_batch_device(pastila_series* h, const int32_t* m_list, int32_t n_m,
                                             pastila_mparams rule, void* const* D_dev, double* D_max_dev);

/* Status of the handle's tile work enqueued so far, for callers of the
 * enqueue-only entry points: call it after the handle's stream has been
 * synchronised.  Returns PASTILA_ETIMEOUT (and clears the flag) if a tile's
 * bounded staging wait ran out since the last check, in which case the outputs
 * of that work are unspecified; PASTILA_OK otherwise.  Reads one host-mapped
 * word; launches nothing.  Errors: EINVAL (NULL handle). */
pastila_status pastila_stage_status(pastila_series* h);

/* --------------------------------------------- snippets (eqs. 5-8, 16-17) ---- */

/* The K snippets of length m: greedy minimisation of ProfileArea (eqs. 16-17;
 * M starts at +inf, each step picks the unchosen segment minimising
 * sum_p min(M_p, D_s(p)), lowest index on ties, sums in FP64), then nearest-
 * snippet labels (eq. 6, argmin over the K chosen profiles, lowest segment index
 * on ties), frac (eq. 7) and the eq. 8 order (frac descending, then index).
 * out: K records in eq. 8 order (host).
 * labels_out: NULL or P int32 (host): the nearest snippet's segment index per position.
 * snippet_profiles_out: NULL or K * P elements (host, float or double per
 *   precision): the chosen profiles in greedy order.
 * Errors: EINVAL (K < 1 or K > min(S, 64), bad m/ell/k), ENOMEM, ECUDA. */
pastila_status pastila_snippets(pastila_series* h, int32_t m, pastila_mparams mp, int32_t K,
                                pastila_snippet* out, int32_t* labels_out,
                                void* snippet_profiles_out);

/* Greedy decisions of FP32 handles (snippets, select_length).  The FP32
 * profiles are accurate to |rho - rho64| <= 2e-6 cell by cell, i.e.
 * |d^2 - d64^2| <= 4e-6 ell (the FP32 tiles recompute ill-conditioned cells
 * exactly to keep it), so each FP32 area of a greedy step has a bound on its
 * distance from the FP64 area of the paper's definitions.  With on = 1 (the default), a step that leaves
 * more than one segment within those bounds of the smallest FP32 area is
 * decided on FP64 areas of FP64 profile rows (of up to 16 contenders, those with
 * the smallest FP32 areas, and of the segments chosen before), lowest index on
 * ties, so that the chosen segments are those of an FP64 search; area_after of
 * such a step is its FP64 area.  With on = 0 every step is decided on the FP32
 * areas alone.  No effect on FP64 handles.  Errors: EINVAL (NULL handle). */
pastila_status pastila_set_fp64_ties(pastila_series* h, int on);

/* --------------------------------------------- length selection (eq. 18) ---- */

/* PaSTiLa's length criterion over a sweep (Section 4.2, eq. 18): for every m in
 * m_list, the greedy K snippets and
 *     crit(m) = sum over ordered pairs p != q of sum_i |D_{c_p}(i) - D_{c_q}(i)|
 *               / max_{s,i} D_s(i)      (0 when that maximum is 0),
 * then m_best = argmax crit (smallest m on ties).  rule gives ell and k per m
 * (0 fields = the defaults m / 2 and (m + 9) / 10; a non-zero ell is used for
 * every m and must be <= min m).
 * m_best: one int32 (host).  crit_out: NULL or n_m doubles (host, m_list order).
 * best_out: NULL or K snippets of length m_best in eq. 8 order (host).
 * Errors: EINVAL (n_m < 1, a bad m, K < 2 or K > min(floor(n / max m), 64)),
 * ENOMEM, ECUDA. */
pastila_status pastila_select_length(pastila_series* h, const int32_t* m_list, int32_t n_m,
                                     pastila_mparams rule, int32_t K, int32_t* m_best,
                                     double* crit_out, pastila_snippet* best_out);

/* --------------------------------------------- allocation-free variant ---- */

/* The greedy snippet search of pastila_snippets (same kernels, same results),
 * for callers that cannot allocate device memory: code whose device memory
 * belongs to another allocator (a framework's caching pool, a process with a
 * fixed memory partition) or that may not allocate once its hot loop runs.
 * The paper has no counterpart; this is a deployment convenience.
 *
 * Inputs and outputs are the caller's device buffers on the current device:
 *   D_dev            S x P FP32 profile set, row-major (as pastila_profiles_device writes it)
 *   chosen_dev       K int32: the chosen segments in greedy order
 *   area_after_dev   K doubles: ProfileArea after each step
 * The working storage (S areas, the P-point curve M) lives in one fixed device
 * array of the library, 4.125 MiB, that every GPU loading the library holds
 * until the process exits; hence S <= 16384 and P <= 1048576, and larger sizes
 * are rejected with EINVAL.  The call allocates nothing and frees nothing.
 * Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default
 * stream) and the call returns without waiting.  The first call on a device,
 * with that device current, looks up the array's device address; make that
 * first call before any stream capture.  All calls share the one array, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race; order them on one stream or synchronise between them.  The looked-up
 * address is kept per device ordinal for the life of the process: after a
 * cudaDeviceReset on a device the entry point must not be called on it again
 * in that process (it would launch on the stale address).
 * Errors: EINVAL (NULL pointer, S, P or K out of range), ECUDA. */
pastila_status pastila_greedy_noalloc(const float* D_dev, int32_t S, int64_t P, int32_t K,
                                      int32_t* chosen_dev, double* area_after_dev, void* stream);

/* -------------------------------------------------------------- engine ---- */

/* Serving engine (no counterpart in the paper: the paper runs one series at a
 * time).  Jobs are whole select_length problems -- a series, its sweep of
 * lengths m_list, the ell/k rule and K -- submitted from any host thread and
 * run by one scheduler thread with continuous batching on one GPU:
 *   - admission: queued jobs are admitted in submission order (policy SHARE)
 *     or by predicted device time (policy SRPT) while fewer than
 *     max_active_jobs are resident and the job's resident memory (series,
 *     window statistics, K chosen profiles per length, small state) plus its
 *     largest S x P profile set fit in the memory budget; a job that can never
 *     fit is refused by pastila_engine_submit with ENOMEM;
 *   - waves: each wave is one tile launch over segment ranges of every active
 *     job's lengths (the wave's eq. 9 cells are shared among the active jobs
 *     as the policy says), then one batched greedy search (eqs. 16-17) and criterion (eq. 18)
 *     for every length whose profiles are complete, then m_best and the eq. 8
 *     records of every job whose lengths are all done; a profile set lives only
 *     from its first wave to its greedy search;
 *   - overlap: up to max_waves_in_flight waves are queued on the device at
 *     once, and jobs that arrive while waves run join the next wave.
 * A job's results are bit-identical to pastila_select_length on a handle of the
 * engine's precision and device for FP32 (FP64: equal up to the criterion's
 * summation order), whatever other jobs share its waves.  All entry points
 * are thread-safe. */
typedef struct pastila_engine pastila_engine;

/* How a wave's tile work is shared among the active jobs, and the admission order. */
typedef enum {
    PASTILA_POLICY_SHARE = 0, /* admission in submission order; each wave's cells shared among the active
                                 jobs (equally, or weighted by age with age_weight_s) */
    PASTILA_POLICY_SRPT = 1   /* shortest remaining first: queued jobs are admitted in order of their
                                 predicted device time (runtime model below), and each wave goes to the
                                 active job with the least predicted remaining time, then the next */
} pastila_policy;

typedef struct {
    int32_t device;
    pastila_precision prec;
    size_t mem_budget_bytes;     /* device memory the engine may hold; 0: 90 % of the memory free at creation */
    int32_t max_active_jobs;     /* jobs resident at once, 1..256; 0: 32 */
    double wave_ed_cells;        /* eq. 9 cells (halo columns included) per wave; 0: 4e9 */
    int32_t max_waves_in_flight; /* 1..8; 0: 2 */
    int32_t fail_alloc_at;       /* fault injection for tests: the n-th device allocation (1-based) of the
                                    engine reports ENOMEM and fails the job it was for; 0: off */
    double age_weight_s;         /* share of a wave per active job: 0 (default) equal shares; > 0 shares in
                                    proportion to 1 + (time since submission) / age_weight_s, which moves
                                    the engine from processor sharing toward arrival order */
    int32_t policy;              /* pastila_policy; 0: PASTILA_POLICY_SHARE */
    int32_t fp32_greedy;         /* FP32 engines: 0 (default) decides near-tied greedy steps on FP64 areas,
                                    as select_length does (pastila_set_fp64_ties); 1 decides every step on
                                    the FP32 areas alone (no FP64 rows: wave times then depend only on the
                                    wave's work, not on how many steps are near-ties) */
    const char* job_log_path;    /* NULL (default): no log; else a file the engine appends one JSON line to
                                    per job that ends (done, failed or cancelled): id, state, status,
                                    message, n, lengths, K, submit / admit / done times (engine clock, s),
                                    latency, first and last wave, ED and profile cells, memory, the
                                    runtime model's prediction, and m_best of a finished job.  The
                                    engine opens it at creation (EINVAL if it cannot) and closes it when
                                    destroyed; lines are flushed as they are written */
} pastila_engine_config;

typedef enum {
    PASTILA_JOB_QUEUED = 0,
    PASTILA_JOB_ACTIVE = 1,
    PASTILA_JOB_DONE = 2,
    PASTILA_JOB_FAILED = 3,
    PASTILA_JOB_CANCELLED = 4
} pastila_job_state;

typedef struct {
    int32_t state;            /* pastila_job_state */
    int32_t status;           /* OK, or the pastila_status that ended the job */
    double t_submit;          /* engine clock, seconds since pastila_engine_create (steady clock) */
    double t_admit;           /* -1 until admitted */
    double t_done;            /* -1 until final; t_done - t_submit is the job's latency */
    int64_t first_wave;       /* first and last wave that carried the job's work; -1 until set */
    int64_t last_wave;
    double ed_cells;          /* eq. 9 cells of the job's tiles, halo columns included */
    double profile_cells;     /* sum over the sweep of S * P */
    size_t mem_bytes;         /* device memory admission asks for: resident + largest profile set */
    size_t resident_bytes;    /* the part held from admission to the job's last wave */
    double predicted_ms;      /* the runtime model's device time of the whole job, made at submission */
} pastila_job_info;

typedef struct {
    uint64_t submitted, done, failed, cancelled;
    uint64_t waves, launches;  /* waves enqueued; kernel launches they issued */
    double ed_cells;           /* eq. 9 cells of all tile launches */
    double profile_cells;      /* S * P summed over the lengths of the finished jobs */
    double busy_ms;            /* device time of the finished waves (events around each wave) */
    size_t mem_budget, mem_held, mem_peak;
    double now;                /* engine clock */
    uint64_t model_waves;      /* finished waves this engine fed to the runtime model */
    double model_rel_err;      /* mean |predicted - measured| / measured of this engine's wave times,
                                  over the waves predicted by a model with >= 8 observations; -1: none */
} pastila_engine_counters;

/* Creates an engine (its streams, memory pool and scheduler thread) on
 * cfg->device; cfg NULL selects every default.  Errors: EINVAL, ENOMEM, ECUDA. */
pastila_status pastila_engine_create(pastila_engine** out, const pastila_engine_config* cfg);

/* Queues one job; the n host values of T are copied before the call returns.
 * m_list: n_m lengths (1 <= n_m <= 64), each 4 <= m <= n, with the ell/k rule
 * of pastila_mparams; 2 <= K <= min(n / max m, 64).  *job_out receives the
 * job's id.  Errors: EINVAL (arguments, tile does not fit shared memory, engine
 * shutting down), ENOMEM (the job can never fit the budget), ECUDA (the engine
 * stopped after a device error). */
pastila_status pastila_engine_submit(pastila_engine* e, const double* T, int64_t n, const int32_t* m_list,
                                     int32_t n_m, pastila_mparams rule, int32_t K, int64_t* job_out);

/* A multivariate series of d coordinates (Section 3.1; Section 3.2 searches
 * every coordinate on its own):
 * T holds d coordinates of n values each, coordinate c at T + c * n.  Queues
 * d jobs, one per coordinate with the same m_list, rule and K, in one step:
 * every coordinate is checked and planned first and nothing is queued unless
 * all are accepted, and the scheduler sees all d jobs at once, so their tiles
 * share waves (one tile launch per wave for all coordinates) as far as slots
 * and memory allow.  jobs_out[c] receives coordinate c's job id; each is
 * polled, read and released as a job of its own.  Errors as
 * pastila_engine_submit, and EINVAL for d outside 1..4096. */
pastila_status pastila_engine_submit_multi(pastila_engine* e, const double* T, int64_t n, int32_t d,
                                           const int32_t* m_list, int32_t n_m, pastila_mparams rule, int32_t K,
                                           int64_t* jobs_out);

/* Waits up to timeout_ms (0: no wait, < 0: no limit) for the job to reach
 * DONE, FAILED or CANCELLED and fills *info (may be NULL) either way.
 * Returns OK when the job is final, ETIMEOUT when it is not; EINVAL for an
 * unknown or released job. */
pastila_status pastila_engine_poll(pastila_engine* e, int64_t job, int32_t timeout_ms, pastila_job_info* info);

/* Results of a DONE job, as pastila_select_length gives them: m_best, the n_m
 * criterion values (crit_out, may be NULL) and the K records of m_best
 * (best_out, may be NULL).  Errors: EBUSY (not final), ECANCELLED, the job's
 * own error for a FAILED job, EINVAL. */
pastila_status pastila_engine_result(pastila_engine* e, int64_t job, int32_t* m_best, double* crit_out,
                                     pastila_snippet* best_out);

/* Cancels a queued or running job; its memory is returned at the next wave
 * boundary (work already on the device finishes first).  Errors: EINVAL
 * (unknown job, or a job that has finished or is in its final wave). */
pastila_status pastila_engine_cancel(pastila_engine* e, int64_t job);

/* Forgets a final job and its results.  Errors: EBUSY (not final), EINVAL. */
pastila_status pastila_engine_release(pastila_engine* e, int64_t job);

/* Engine counters.  Errors: EINVAL. */
pastila_status pastila_engine_stats(pastila_engine* e, pastila_engine_counters* out);

/* Lets the waves on the device finish, cancels every other job, stops the
 * scheduler and frees everything.  NULL is a no-op. */
void pastila_engine_destroy(pastila_engine* e);

/* ------------------------------------------------------- runtime model ---- */

/* Section 4.2 predicts the run time of the search for each snippet length
 * with a polynomial regression trained on earlier runs.  Here one such model
 * per precision (process-wide, shared by every engine) predicts device time:
 *   ms = c0 E + c1 E x + c2 E x^2 + c3 G + c4 w
 * with E the eq. 9 cells of the tile work in units of 1e9 (halo columns
 * included) at length m, x = m / 256 (summed over the lengths), G the GB of
 * profile set the greedy search reads (K passes over S x P values per length)
 * and w the number of engine waves.  Every finished engine wave is one
 * observation (its features, its time between events around it); the
 * coefficients are the least-squares fit to all observations so far, each
 * pulled toward a prior by a ridge term of 1e-4 times its own diagonal entry
 * of the normal matrix (plus 1e-9), so that directions the data does not
 * determine (every wave at one length) keep the prior's values.  The engine's SRPT policy and
 * pastila_job_info.predicted_ms use it.  Not thread-affine; all calls are
 * thread-safe. */
typedef struct {
    int32_t prec;        /* pastila_precision of the model */
    int32_t n_coef;      /* 5 */
    double coef[5];      /* c0 .. c4 as above (ms) */
    double prior[5];     /* the ridge term's target */
    double xtx[25];      /* normal equations of the observations so far: sum f f^T (row-major) */
    double xty[5];       /* sum f * ms */
    uint64_t observations;
    uint64_t err_count;  /* observations predicted by the model after >= 8 observations */
    double rel_err;      /* their mean |predicted - measured| / measured; -1 when err_count is 0 */
} pastila_runtime_model;

/* Copies the model of prec.  Errors: EINVAL. */
pastila_status pastila_model_get(pastila_precision prec, pastila_runtime_model* out);

/* Replaces the model of in->prec by in's prior and normal equations (a warm
 * start from an earlier process's pastila_model_get) and refits; coef, the
 * error fields and n_coef are ignored.  Errors: EINVAL (n_coef != 5, a
 * non-finite entry, unknown precision). */
pastila_status pastila_model_set(const pastila_runtime_model* in);

/* Adds one observation: features f[5] = {E, E x, E x^2, G, w} as above and its
 * measured time ms > 0 (for callers that time their own runs).  Errors: EINVAL. */
pastila_status pastila_model_observe(pastila_precision prec, const double* f, double ms);

/* Forgets every observation of prec (coefficients back to the prior).  Errors: EINVAL. */
pastila_status pastila_model_reset(pastila_precision prec);

/* Predicted device time (ms) of one job as the engine plans it: its lengths'
 * tile cells under the tile layouts chosen for smem_limit bytes of shared
 * memory per CTA (pastila_plan_layout), K greedy passes per length and one
 * wave per wave_ed_cells of tile work (0: 4e9).  Host code only.  Errors:
 * EINVAL (arguments as pastila_engine_submit, no layout fits). */
pastila_status pastila_model_predict(pastila_precision prec, int64_t n, const int32_t* m_list, int32_t n_m,
                                     pastila_mparams rule, int32_t K, size_t smem_limit, double wave_ed_cells,
                                     double* ms_out);

/* The greedy snippet search of pastila_snippets without materialising the S x P
 * profile set, for lengths whose D does not fit the budget or the device
 * (pastila_snippets switches to it by itself when allocating D fails with
 * ENOMEM).  Rows of D are recomputed by the profile kernel: one pass over all
 * segments, which also keeps a sketch of every row (per block of whole tiles:
 * its sum, largest and smallest value), then, at every step, only the rows
 * whose lower area bound can still beat the best (from the sketch against the
 * current curve M, and, for a row recomputed earlier, its block areas then
 * less the block's drop in M since); a step whose bounds leave more than half
 * of the segments open makes one more pass instead.  It uses the tile layout
 * pastila_snippets uses.  Memory: K + 10 rows of P values and P doubles, at
 * most 256 MiB of per-tile partials and 512 MiB of sketches and block areas
 * (the blocks are as fine as that allows, down to one tile).  Results
 * (records, labels, chosen profiles) are
 * identical to pastila_snippets on the materialised D: every area it compares
 * is computed exactly as there.  work_out (may be NULL) receives two values:
 * full passes over the segments and rows recomputed.  No counterpart in the
 * paper (Section 4.2 materialises D over a cluster).  Errors as
 * pastila_snippets. */
pastila_status pastila_snippets_streamed(pastila_series* h, int32_t m, pastila_mparams mp, int32_t K,
                                         pastila_snippet* out, int32_t* labels_out, void* snippet_profiles_out,
                                         int64_t* work_out);

/* ----------------------------------------------------------- autotuner ---- */

/* The tile layout of a length (positions per CTA W, row groups NG, threads NT,
 * lanes per selection run GS, always 32: one warp per run of positions) comes
 * from a cost model unless the autotuner
 * has chosen one.  pastila_tune times, for every m of m_list with the ell/k
 * rule, the model's layout and up to max_candidates - 1 rivals (the model's
 * best two- and four-CTA cluster layouts and its best layout of at most 256
 * threads and half an SM's shared memory, so that two CTAs share an SM; then
 * the cheapest of every thread count, then by modelled cost, these within
 * 1.5x of the model's best), on the first min(S, 64) segments of h's series, and keeps the fastest (a rival must beat
 * the layout kept so far by more than 1 %, so that layouts within timing noise
 * of each other do not trade places from run to run) in a process-wide
 * table keyed by (precision, m, ell, k) that every later call uses (handles and
 * engines alike; a captured select_length graph is rebuilt).  Results depend
 * on the layout only through FP32 rounding (the seeds sit at the tile and
 * row-group edges); a given layout always gives the same results.  out, when
 * not NULL, receives n_m records.  No counterpart in the paper, whose kernel
 * has one fixed layout.  Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct {
    int32_t m;
    int32_t W, NG, NT;     /* the chosen layout */
    int32_t GS;            /* lanes per k-th selection run (32) */
    int32_t CS;            /* CTAs per tile: 1, 2 or 4 (a thread-block cluster splitting the rows) */
    int32_t candidates;    /* layouts timed */
    double ms_model;       /* device time of the cost model's layout on the sample */
    double ms_best;        /* device time of the chosen layout */
} pastila_tune_result;

pastila_status pastila_tune(pastila_series* h, const int32_t* m_list, int32_t n_m, pastila_mparams rule,
                            int32_t max_candidates, pastila_tune_result* out);

/* Forgets every tuned layout (the cost model decides again). */
void pastila_tune_clear(void);

/* Writes (pastila_tune_set) or reads (pastila_tune_get) one entry of the tuned
 * table: for (prec, m, ell, k), tile width W (a multiple of 32), NG row groups
 * asked per CTA, GS lanes per selection run (must be 32: the selection runs one
 * warp per run of positions), CS CTAs per tile (1, 2 or 4).  A table saved with
 * pastila_tune_get and restored with pastila_tune_set reproduces the tuned
 * runs' results bit for bit.  A layout that does not fit the device's shared
 * memory is ignored when it is looked up (the cost model decides instead).
 * Errors: EINVAL (out of range; get: no entry). */
pastila_status pastila_tune_set(pastila_precision prec, int32_t m, int32_t ell, int32_t k, int32_t W, int32_t NG,
                                int32_t GS, int32_t CS);
pastila_status pastila_tune_get(pastila_precision prec, int32_t m, int32_t ell, int32_t k, int32_t* W, int32_t* NG,
                                int32_t* GS, int32_t* CS);

/* The tile layout that h's calls use for length m with mp: out5 = {W, NG (row
 * groups per CTA), NT (threads per CTA), GS, CS}.  Errors: EINVAL. */
pastila_status pastila_tile_layout(pastila_series* h, int32_t m, pastila_mparams mp, int32_t* out5);

/* The same choice without a device (host code only): the tuned table's entry
 * if it fits smem_limit bytes of dynamic shared memory per CTA, else the cost
 * model's layout for a series of n values.  out8 = {W, NG, NT, GS, CS, Rg (rows
 * per group), Rh (rows per CTA), shared-memory bytes}.  Errors: EINVAL (no
 * layout fits). */
pastila_status pastila_plan_layout(pastila_precision prec, int64_t n, int32_t m, pastila_mparams mp,
                                   size_t smem_limit, int32_t* out8);

/* ------------------------------------------------------------- tracing ---- */

/* Kernel launches the handle has issued since it was created. */
uint64_t pastila_kernel_launches(const pastila_series* h);

/* Turns per-launch timing of the profile tile kernel on (1) or off (0).  While
 * on, every launch is bracketed by CUDA events on the handle's stream; the
 * accumulated device time is read (after the stream is idle) with
 * pastila_tile_time.  Errors: EINVAL, ECUDA. */
pastila_status pastila_set_timing(pastila_series* h, int on);

/* Total device milliseconds and number of timed launches of the profile tile
 * kernel since timing was turned on, and the ED cells (entries of the eq. 9
 * matrix, the halo columns of each tile included) those launches computed.
 * Waits for the handle's stream.  Any output may be NULL. */
pastila_status pastila_tile_time(pastila_series* h, double* ms, int64_t* launches, double* ed_cells);

/* -------------------------------------------------------------- probe ---- */

/* Measured fused multiply-add rates of `device`, in TFLOP/s (2 FLOP per FMA):
 * a kernel of eight independent FMA chains per thread over 8 CTAs of 256
 * threads per SM (148 x 8 on a B300), timed with events after a warm-up launch, in FP32 and in FP64.
 * The roofline of the profile kernel, which is bound by FP32/integer issue
 * rather than by memory or tensor cores, can be read against these.  No
 * counterpart in the paper.  Allocates and frees a small output buffer.
 * Errors: EINVAL, ECUDA. */
pastila_status pastila_probe_fma(int32_t device, double* fp32_tflops, double* fp64_tflops);

#ifdef __cplusplus
}
#endif
#endif /* PASTILA_H_ */
