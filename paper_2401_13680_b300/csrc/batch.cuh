// Batched launches: every length m of a sweep (and, in the engine, every job of
// a wave) is one item; one launch of each kernel covers all items.
//
//   tiles      one flattened grid: CTA b belongs to the item whose CTA range
//              [cta_begin, cta_begin + S * ntiles * CS) contains b (CS = 2: the
//              launch has clusters of two CTAs, one per half of a tile's rows)
//   greedy     per step t, one 2-D grid (segments x items) for the areas, one
//              CTA per item for the argmin, one 2-D grid for the curve update
//   criterion  one 2-D grid of partial sums, one thread per item to finish
// The arithmetic is the single-item one (tile.cuh, snippets.cuh); only the
// mapping from blocks to items is new, so a batched result is bit-identical to
// the same item run alone.
#pragma once
#include <cstdint>

#include "keys.cuh"
#include "snippets.cuh"
#include "tile.cuh"

namespace pastila {

// FP64 re-evaluation of near-tied greedy steps (FP32 items).  The FP32 profiles
// are accurate to |d rho| <= 2e-6 cell by cell (the tolerance rule's bound
// below d_floor, which the FP32 tiles meet at every cell: they recompute the
// ill-conditioned ones exactly), hence every FP32 area of a step is within
// E_s = sum_p b(min(M_p, D_s(p))) of the FP64 area the oracle computes, b the
// per-value bound of row_bound_partial.
// When more segments than the FP32 minimum lie within the bounds of it, the
// step is decided on FP64 areas: FP64 rows of those contenders (at most
// REF_NCAND, those with the smallest FP32 areas) and of every earlier chosen
// segment come from the FP64 tile kernel, and the curve M of FP64 rows gives
// the FP64 areas (lowest segment index on ties).
constexpr int REF_NCAND = 16;
// layout of an item's refinement state (int32):
constexpr int REF_TODO_N = 0;      // rows the next FP64 row launch computes
constexpr int REF_NC = 1;          // contenders of the current step (0: decided in FP32)
constexpr int REF_PARTIAL = 2;     // bit c: contender c's FP64 row skips tiles (see batched_refine_need_kernel)
constexpr int REF_DROPPED = 3;     // 1: some tile is needed by no contender; the areas compared leave it out
constexpr int REF_HAS = 4;         // [64]: 1 when rows64 slot t holds chosen segment t's FP64 row
constexpr int REF_TODO_SEG = 68;   // [64 + REF_NCAND]: segments of the to-do rows
constexpr int REF_TODO_SLOT = REF_TODO_SEG + 64 + REF_NCAND;  // and their rows64 slots
constexpr int REF_CAND = REF_TODO_SLOT + 64 + REF_NCAND;       // [REF_NCAND] contenders, ascending index
constexpr int REF_STATE_INTS = REF_CAND + REF_NCAND;

template <typename real>
struct BatchItem {
    ProfileArgs<real> A;   // profile arguments (series, statistics, D, D max key)
    TileGeom G;            // tile layout of this item
    // FP64 re-evaluation (rows64 == nullptr: off): FP64 profile arguments of
    // the same length (their D is rows64; their D max key a scratch word), the
    // FP64 tile layout, (K + REF_NCAND) x P FP64 rows (slot t < K: chosen
    // segment t; slot K + c: contender c), the S FP32 area bounds of the step,
    // the contenders' FP64 areas, the state above and the constant c of
    // row_bound_partial (2.2 ell times 2e-6)
    ProfileArgs<double> A64;
    TileGeom G64;
    double* rows64;
    float* bound;
    double* cand_area;
    uint8_t* need;         // [REF_NCAND][A64.ntiles]: 1 where contender c's FP64 tile is computed
    int32_t* rst;
    float bc;
    long long cta_begin;   // first CTA of this item in the flattened tile grid (even for cluster tiles)
    long long ctas;        // its CTA count (CTAs past it, alignment padding, do nothing)
    int s_begin;           // first segment of this launch's share of the item (the
                           // engine splits an item's segments over several waves)
    real* M;               // representativeness curve, P values
    double* area;          // S areas of the current greedy step
    int32_t* chosen;       // K chosen segments, greedy order
    double* area_after;    // K areas
    double* crit_part;     // CRIT_BLOCKS partial sums of the eq. 18 numerator
    double* crit;          // eq. 18 value
    int K;
};

constexpr int CRIT_BLOCKS = 64;

template <typename real, int V>
__global__ void __launch_bounds__(512) batched_tiles_kernel(const BatchItem<real>* __restrict__ items, int n) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ProfileArgs<real> sA;
    __shared__ TileGeom sG;
    __shared__ long long s_first, s_ctas;
    __shared__ int s_sbegin;
    static_assert(sizeof(ProfileArgs<real>) % 4 == 0 && sizeof(TileGeom) % 4 == 0, "copied as 4-byte words");
    const long long b = blockIdx.x;
    // the item of this CTA: the last one whose first CTA is at or before it (the
    // first item starts at CTA 0).  Up to 32 items, warp 0 reads every item's
    // first CTA at once and copies the item's arguments word by word, so the CTA
    // waits for two rounds of loads instead of a chain of them
    if (n <= 32) {
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            const unsigned m = __ballot_sync(0xffffffffu, l < n && items[l].cta_begin <= b);
            const int lo = 31 - __clz(m);
            const uint32_t* srcA = reinterpret_cast<const uint32_t*>(&items[lo].A);
            uint32_t* dstA = reinterpret_cast<uint32_t*>(&sA);
            for (int w = l; w < (int)(sizeof(ProfileArgs<real>) / 4); w += 32) dstA[w] = srcA[w];
            const uint32_t* srcG = reinterpret_cast<const uint32_t*>(&items[lo].G);
            uint32_t* dstG = reinterpret_cast<uint32_t*>(&sG);
            for (int w = l; w < (int)(sizeof(TileGeom) / 4); w += 32) dstG[w] = srcG[w];
            if (l == 0) {
                s_first = items[lo].cta_begin;
                s_ctas = items[lo].ctas;
                s_sbegin = items[lo].s_begin;
            }
        }
    } else if (threadIdx.x == 0) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].cta_begin <= b) lo = mid; else hi = mid - 1;
        }
        sA = items[lo].A;
        sG = items[lo].G;
        s_first = items[lo].cta_begin;
        s_ctas = items[lo].ctas;
        s_sbegin = items[lo].s_begin;
    }
    __syncthreads();
    const long long local = b - s_first;
    if (local >= s_ctas) return;  // padding: its cluster partner is a one-CTA tile
    const int cs = sG.CS;  // an item of cluster tiles starts at an even CTA of a cluster launch
    const long long per_seg = (long long)sA.ntiles * cs;
    const int s = s_sbegin + (int)(local / per_seg), tt = (int)((local % per_seg) / cs);
    profile_tile<real, V>(sA, sG, s, tt, smem);
}

// areas of greedy step t for every item: grid (max S, n items)
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS) batched_area_kernel(const BatchItem<real>* __restrict__ items, int t) {
    __shared__ double red[AREA_THREADS / 32];
    const BatchItem<real>& it = items[blockIdx.y];
    const int s = blockIdx.x;
    const int S = it.A.S;
    if (s >= S || t >= it.K) return;
    const int64_t P = it.A.P;
    bool skip = false;
    for (int u = 0; u < t; ++u) skip |= it.chosen[u] == s;
    if (skip) {
        if (threadIdx.x == 0) it.area[s] = __longlong_as_double(0x7ff0000000000000ll);
        return;
    }
    const real* row = it.A.D + (int64_t)s * P;
    const real* M = t == 0 ? (const real*)nullptr : it.M;
    const double tot = block_sum(row_min_partial(row, M, P), red);
    if (threadIdx.x == 0) it.area[s] = tot;
    if (it.rows64) {  // the error bound of this area (FP32 items with refinement), 2 % margin
        const double e = block_sum((double)row_bound_partial(row, M, P, it.bc), red);
        if (threadIdx.x == 0) it.bound[s] = (float)(1.02 * e);
    }
}

// The greedy choice of step t for every item (one CTA of 1024 per item): the
// FP32 argmin (lowest index on ties), exactly as batched_argmin_kernel.  Items
// with refinement then count the contenders, the unchosen segments whose FP32
// area is within the two error bounds (and a 1e-9 relative margin for the
// rounding of the FP64 sums) of the minimum; one contender decides the step
// here; otherwise up to REF_NCAND contenders with the smallest FP32 areas
// (lowest index on ties) and every earlier chosen segment without an FP64 row go
// on the to-do list of the FP64 row launch, and batched_choose_update_kernel
// decides.
template <typename real>
__global__ void batched_select_kernel(const BatchItem<real>* __restrict__ items, int t) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    __shared__ int picked[REF_NCAND];
    const BatchItem<real>& it = items[blockIdx.x];
    if (t >= it.K) return;
    const int S = it.A.S;
    const int tid = threadIdx.x;
    auto chosen_before = [&](int s) {
        bool c = false;
        for (int u = 0; u < t; ++u) c |= it.chosen[u] == s;
        return c;
    };
    // block argmin of key(s) over the segments admit(s) accepts (lowest index on ties)
    auto block_argmin = [&](auto&& key, auto&& admit, double* bestv) {
        double best = __longlong_as_double(0x7ff0000000000000ll);
        int bidx = 0x7fffffff;
        for (int s = tid; s < S; s += blockDim.x) {
            if (!admit(s)) continue;
            const double a = key(s);
            if (a < best || (a == best && s < bidx)) {
                best = a;
                bidx = s;
            }
        }
        bv[tid] = best;
        bi[tid] = bidx;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (tid < w) {
                const double ov = bv[tid + w];
                const int oi = bi[tid + w];
                if (ov < bv[tid] || (ov == bv[tid] && oi < bi[tid])) {
                    bv[tid] = ov;
                    bi[tid] = oi;
                }
            }
            __syncthreads();
        }
        const int r = bi[0];
        *bestv = bv[0];
        __syncthreads();
        return r;
    };
    double Ab;
    const int b = block_argmin([&](int s) { return it.area[s]; }, [&](int s) { return !chosen_before(s); }, &Ab);
    if (!it.rows64) {
        if (tid == 0) {
            it.chosen[t] = b;
            it.area_after[t] = Ab;
        }
        return;
    }
    int32_t* rst = it.rst;
    if (t == 0) {  // a new search: no chosen segment has an FP64 row yet
        for (int u = tid; u < 64; u += blockDim.x) rst[REF_HAS + u] = 0;
        __syncthreads();
    }
    const double Eb = (double)it.bound[b];
    auto contender = [&](int s) {
        return !chosen_before(s) && it.area[s] - Ab <= Eb + (double)it.bound[s] + 1e-9 * Ab;
    };
    int cnt = 0;
    for (int s = tid; s < S; s += blockDim.x) cnt += contender(s) ? 1 : 0;
    bi[tid] = cnt;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (tid < w) bi[tid] += bi[tid + w];
        __syncthreads();
    }
    cnt = bi[0];
    __syncthreads();
    if (cnt <= 1) {
        if (tid == 0) {
            it.chosen[t] = b;
            it.area_after[t] = Ab;
            rst[REF_TODO_N] = 0;
            rst[REF_NC] = 0;
            rst[REF_PARTIAL] = 0;
            rst[REF_DROPPED] = 0;
            rst[REF_HAS + t] = 0;
        }
        return;
    }
    const int nc = cnt < REF_NCAND ? cnt : REF_NCAND;
    for (int c = 0; c < nc; ++c) {
        double v;
        const int s = block_argmin([&](int q) { return it.area[q]; },
                                   [&](int q) {
                                       if (!contender(q)) return false;
                                       for (int u = 0; u < c; ++u)
                                           if (picked[u] == q) return false;
                                       return true;
                                   },
                                   &v);
        if (tid == 0) picked[c] = s;
        __syncthreads();
    }
    if (tid == 0) {
        for (int i = 1; i < nc; ++i) {  // ascending segment index
            const int x = picked[i];
            int j = i - 1;
            while (j >= 0 && picked[j] > x) {
                picked[j + 1] = picked[j];
                --j;
            }
            picked[j + 1] = x;
        }
        int n = 0;
        for (int u = 0; u < t; ++u) {
            if (!rst[REF_HAS + u]) {
                rst[REF_TODO_SEG + n] = it.chosen[u];
                rst[REF_TODO_SLOT + n] = u;
                rst[REF_HAS + u] = 1;  // filled by the row launch that follows
                ++n;
            }
        }
        for (int c = 0; c < nc; ++c) {
            rst[REF_CAND + c] = picked[c];
            rst[REF_TODO_SEG + n] = picked[c];
            rst[REF_TODO_SLOT + n] = it.K + c;
            ++n;
        }
        rst[REF_TODO_N] = n;
        rst[REF_NC] = nc;
        rst[REF_PARTIAL] = 0;
        rst[REF_DROPPED] = 0;
        rst[REF_HAS + t] = 0;
    }
}

// Which FP64 tiles of the contenders' rows a step needs.  From step 1 on, where
// a contender's FP32 value less its error bound is at least the FP32 curve plus
// its bound, at every position of a tile, the FP64 value there is at least the
// FP64 curve M64 (each FP32 value is within value_bound of its FP64 value, and
// M64 <= the chosen row that attains the FP32 curve), so min(M64, D64) = M64 on
// the whole tile and its FP64 values are not needed; the tile is skipped and
// the area sums take M64 there.  A tile that no contender needs adds the same
// sum of M64 to every contender's area, so the comparison leaves it out and the
// chosen segments' FP64 rows are computed only on the tiles some contender
// needs (row REF_NCAND of the flags).  At step 0 (M = +inf) every tile is
// needed.  Grid (largest FP64 tile count, n items), NEED_THREADS threads.
constexpr int NEED_THREADS = 256;
template <typename real>
__global__ void __launch_bounds__(NEED_THREADS) batched_refine_need_kernel(const BatchItem<real>* __restrict__ items,
                                                                           int t) {
    const BatchItem<real>& it = items[blockIdx.y];
    if (t >= it.K || !it.rows64) return;
    const int nc = it.rst[REF_NC];
    const int nt = it.A64.ntiles, W = it.A64.W;
    const int tile = blockIdx.x;
    if (nc == 0 || tile >= nt) return;
    const int64_t P = it.A.P;
    const int64_t p0 = (int64_t)tile * W;
    const int64_t p1 = p0 + W < P ? p0 + W : P;
    bool any = false;
    for (int c = 0; c < nc; ++c) {
        bool need = t == 0;
        if (!need) {
            const real* row = it.A.D + (int64_t)it.rst[REF_CAND + c] * P;
            for (int64_t p = p0 + threadIdx.x; p < p1 && !need; p += NEED_THREADS) {
                const float d = (float)row[p], mm = (float)it.M[p];
                need = d - 1.02f * value_bound(d, it.bc) < mm + 1.02f * value_bound(mm, it.bc) + 1e-5f * (1.0f + mm);
            }
        }
        need = __syncthreads_or(need);
        any |= need;
        if (threadIdx.x == 0) {
            it.need[c * nt + tile] = need ? 1 : 0;
            if (!need) atomicOr(&it.rst[REF_PARTIAL], 1 << c);
        }
    }
    if (threadIdx.x == 0) {
        it.need[REF_NCAND * nt + tile] = any ? 1 : 0;
        if (!any) it.rst[REF_DROPPED] = 1;
    }
}

// FP64 rows of an item's to-do list (one item per launch): grid (ntiles64 CS64,
// K + REF_NCAND, at least the longest to-do list); each CTA computes tile
// blockIdx.x / CS64 of to-do row blockIdx.y (CTAs past the list's end return at
// once).  Row y goes to rows64 slot todo_slot[y] (the profile tile writes row
// s - row_base of its D).
template <int V>
__global__ void __launch_bounds__(512) refine_rows_kernel(const BatchItem<float>* __restrict__ item, int t) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ProfileArgs<double> sA;
    __shared__ TileGeom sG;
    if (t >= item->K || !item->rows64) return;
    const int32_t* rst = item->rst;
    const int n = rst[REF_TODO_N];
    if ((int)blockIdx.y >= n) return;
    if (threadIdx.x == 0) {
        sA = item->A64;
        sG = item->G64;
    }
    __syncthreads();
    const int seg = rst[REF_TODO_SEG + blockIdx.y], slot = rst[REF_TODO_SLOT + blockIdx.y];
    const int tile = (int)blockIdx.x / sG.CS;
    // a tile the step does not need: a contender's skipped tile, or one no contender needs
    if (!item->need[(slot >= item->K ? slot - item->K : REF_NCAND) * sA.ntiles + tile]) return;
    profile_tile<double, V>(sA, sG, seg, tile, smem, seg - slot);
}

// FP64 areas of the contenders of step t: cand_area[c] = sum_p min(M64_p,
// row64_c(p)), M64 = the minimum of the FP64 rows of the chosen segments 0 .. t-1
// (+inf at step 0).  Grid (REF_NCAND, n items), AREA_THREADS threads.
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS) batched_refine_area_kernel(const BatchItem<real>* __restrict__ items,
                                                                           int t) {
    __shared__ double red[AREA_THREADS / 32];
    const BatchItem<real>& it = items[blockIdx.y];
    const int c = blockIdx.x;
    if (t >= it.K || !it.rows64 || c >= it.rst[REF_NC]) return;
    const int64_t P = it.A.P;
    const double* R64 = it.rows64;
    const double* row = R64 + (int64_t)(it.K + c) * P;
    const uint8_t* nd = it.need + (size_t)c * it.A64.ntiles;  // skipped tiles: min(M64, D64) = M64
    const uint8_t* any = it.need + (size_t)REF_NCAND * it.A64.ntiles;  // tiles no contender needs: left out
    const int W64 = it.A64.W;
    double a0 = 0.0, a1 = 0.0;
    int64_t p = threadIdx.x;
    auto term = [&](int64_t q) {
        const int tq = (int)(q / W64);
        if (!any[tq]) return 0.0;
        double v = nd[tq] ? row[q] : __longlong_as_double(0x7ff0000000000000ll);
        for (int u = 0; u < t; ++u) {
            const double w = R64[(int64_t)u * P + q];
            v = w < v ? w : v;
        }
        return v;
    };
    for (; p + AREA_THREADS < P; p += 2 * AREA_THREADS) {
        a0 += term(p);
        a1 += term(p + AREA_THREADS);
    }
    for (; p < P; p += AREA_THREADS) a0 += term(p);
    const double tot = block_sum(a0 + a1, red);
    if (threadIdx.x == 0) it.cand_area[c] = tot;
}

// Decides a step that went to FP64 (the smallest FP64 area, lowest segment index
// on ties: the contenders are in ascending index order), keeps the chosen
// segment's FP64 row in slot t, and updates the FP32 curve M <- min(M, D_chosen)
// (not after the last step).  Every CTA takes the decision itself.  Grid
// (ceil(max P / 256), n items).
template <typename real>
__global__ void batched_choose_update_kernel(const BatchItem<real>* __restrict__ items, int t) {
    const BatchItem<real>& it = items[blockIdx.y];
    if (t >= it.K) return;
    const int64_t P = it.A.P;
    const bool refined = it.rows64 && it.rst[REF_NC] > 0;
    int seg, best = 0;
    if (refined) {
        const int nc = it.rst[REF_NC];
        for (int c = 1; c < nc; ++c)
            if (it.cand_area[c] < it.cand_area[best]) best = c;
        seg = it.rst[REF_CAND + best];
    } else {
        seg = it.chosen[t];
    }
    if (refined && blockIdx.x == 0 && threadIdx.x == 0) {
        it.chosen[t] = seg;
        // the FP64 area when every tile was summed, else the FP32 one (within the
        // FP32 rule of it); the chosen segment's FP64 row is complete unless tiles
        // were skipped (then a later step computes it again)
        const bool dropped = it.rst[REF_DROPPED] != 0;
        it.area_after[t] = dropped ? it.area[seg] : it.cand_area[best];
        it.rst[REF_HAS + t] = dropped || ((it.rst[REF_PARTIAL] >> best) & 1) ? 0 : 1;
        if (dropped) {  // the chosen rows this step computed cover only the tiles it needed
            const int nt = it.rst[REF_TODO_N];
            for (int y = 0; y < nt; ++y) {
                const int slot = it.rst[REF_TODO_SLOT + y];
                if (slot < it.K) it.rst[REF_HAS + slot] = 0;
            }
        }
    }
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    if (refined) it.rows64[(int64_t)t * P + p] = it.rows64[(int64_t)(it.K + best) * P + p];
    if (t + 1 < it.K) {
        const real d = it.A.D[(int64_t)seg * P + p];
        if (t == 0) {
            it.M[p] = d;
        } else {
            const real mm = it.M[p];
            it.M[p] = d < mm ? d : mm;
        }
    }
}

// argmin of step t for every item: one CTA of 1024 per item
template <typename real>
__global__ void batched_argmin_kernel(const BatchItem<real>* __restrict__ items, int t) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    const BatchItem<real>& it = items[blockIdx.x];
    if (t >= it.K) return;
    const int S = it.A.S;
    double best = __longlong_as_double(0x7ff0000000000000ll);
    int bidx = 0x7fffffff;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double a = it.area[s];
        bool chosen_already = false;
        for (int u = 0; u < t; ++u) chosen_already |= it.chosen[u] == s;
        if (chosen_already) continue;
        if (a < best || (a == best && s < bidx)) { best = a; bidx = s; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const double ov = bv[threadIdx.x + w];
            const int oi = bi[threadIdx.x + w];
            if (ov < bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        it.chosen[t] = bi[0];
        it.area_after[t] = bv[0];
    }
}

// M <- min(M, D_{chosen[t]}) for every item: grid (ceil(max P / 256), n items)
template <typename real>
__global__ void batched_update_kernel(const BatchItem<real>* __restrict__ items, int t) {
    const BatchItem<real>& it = items[blockIdx.y];
    const int64_t P = it.A.P;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || t + 1 >= it.K) return;
    const real d = it.A.D[(int64_t)it.chosen[t] * P + p];
    if (t == 0) {
        it.M[p] = d;
    } else {
        const real mm = it.M[p];
        it.M[p] = d < mm ? d : mm;
    }
}

// eq. 18 numerator partial sums: grid (CRIT_BLOCKS, n items)
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS) batched_criterion_kernel(const BatchItem<real>* __restrict__ items) {
    __shared__ double red[AREA_THREADS / 32];
    const BatchItem<real>& it = items[blockIdx.y];
    const int64_t P = it.A.P;
    const real* D = it.A.D;
    const int K = it.K;
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * AREA_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * AREA_THREADS + threadIdx.x; i < P; i += stride) {
        for (int a = 0; a < K; ++a) {
            const double x = (double)D[(int64_t)it.chosen[a] * P + i];
            for (int b = a + 1; b < K; ++b) {
                const double y = (double)D[(int64_t)it.chosen[b] * P + i];
                acc += fabs(x - y);
            }
        }
    }
    const double tot = block_sum(2.0 * acc, red);
    if (threadIdx.x == 0) it.crit_part[blockIdx.x] = tot;
}

// crit = sum of the partials / D max, one thread per item; then m_best over the
// items in [0, n) (smallest m on ties) into best_idx.  One CTA.
template <typename real>
__global__ void batched_finish_kernel(const BatchItem<real>* __restrict__ items, int n, int32_t* __restrict__ best_idx) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const BatchItem<real>& it = items[i];
        double num = 0.0;
        for (int b = 0; b < CRIT_BLOCKS; ++b) num += it.crit_part[b];
        const double den = KeyOf<double>::dec(*it.A.dmax_key);
        *it.crit = den > 0.0 ? num / den : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0 && best_idx) {
        int b = 0;
        for (int i = 1; i < n; ++i) {
            const double ci = *items[i].crit, cb = *items[b].crit;
            if (ci > cb || (ci == cb && items[i].A.m < items[b].A.m)) b = i;
        }
        *best_idx = b;
    }
}

// nearest-snippet counts for the item best_idx selects (or item 0 when NULL):
// grid (ceil(max P / 256)); counts[] must start at 0
template <typename real>
__global__ void batched_neighbors_kernel(const BatchItem<real>* __restrict__ items, const int32_t* __restrict__ best_idx,
                                         int32_t* __restrict__ labels, unsigned long long* __restrict__ counts) {
    __shared__ unsigned int local[64];
    const BatchItem<real>& it = items[best_idx ? *best_idx : 0];
    if (threadIdx.x < 64) local[threadIdx.x] = 0;
    __syncthreads();
    const int64_t P = it.A.P;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int K = it.K;
    if (p < P) {
        int bt = 0;
        real bv = it.A.D[(int64_t)it.chosen[0] * P + p];
        for (int t = 1; t < K; ++t) {
            const real v = it.A.D[(int64_t)it.chosen[t] * P + p];
            if (v < bv || (v == bv && it.chosen[t] < it.chosen[bt])) { bv = v; bt = t; }
        }
        if (labels) labels[p] = it.chosen[bt];
        atomicAdd(&local[bt], 1u);
    }
    __syncthreads();
    if ((int)threadIdx.x < K && local[threadIdx.x])
        atomicAdd(&counts[threadIdx.x], (unsigned long long)local[threadIdx.x]);
}

// eq. 8 records of the item best_idx selects.  One thread.
template <typename real>
__global__ void batched_records_kernel(const BatchItem<real>* __restrict__ items, const int32_t* __restrict__ best_idx,
                                       const unsigned long long* __restrict__ counts, int32_t* __restrict__ out_index,
                                       int32_t* __restrict__ out_rank, double* __restrict__ out_frac,
                                       double* __restrict__ out_area) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const BatchItem<real>& it = items[best_idx ? *best_idx : 0];
    const int K = it.K;
    int order[64];
    for (int t = 0; t < K; ++t) order[t] = t;
    for (int i = 1; i < K; ++i) {
        const int x = order[i];
        int j = i - 1;
        while (j >= 0) {
            const int y = order[j];
            const bool before = counts[x] > counts[y] || (counts[x] == counts[y] && it.chosen[x] < it.chosen[y]);
            if (!before) break;
            order[j + 1] = y;
            --j;
        }
        order[j + 1] = x;
    }
    for (int i = 0; i < K; ++i) {
        const int t = order[i];
        out_index[i] = it.chosen[t];
        out_rank[i] = t;
        out_frac[i] = (double)counts[t] / (double)it.A.P;
        out_area[i] = it.area_after[t];
    }
}

template <typename real>
__global__ void batched_init_dmax_kernel(const BatchItem<real>* __restrict__ items, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) *items[i].A.dmax_key = KeyOf<double>::enc(0.0);
}

}  // namespace pastila
