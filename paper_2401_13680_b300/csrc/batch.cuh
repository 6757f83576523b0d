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

template <typename real>
struct BatchItem {
    ProfileArgs<real> A;   // profile arguments (series, statistics, D, D max key)
    TileGeom G;            // tile layout of this item
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
    const long long b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].cta_begin <= b) lo = mid; else hi = mid - 1;
    }
    if (threadIdx.x == 0) {
        sA = items[lo].A;
        sG = items[lo].G;
    }
    __syncthreads();
    const long long local = b - items[lo].cta_begin;
    if (local >= items[lo].ctas) return;  // padding: its cluster partner is a one-CTA tile
    const int cs = sG.CS;  // an item of cluster tiles starts at an even CTA of a cluster launch
    const long long per_seg = (long long)sA.ntiles * cs;
    const int s = items[lo].s_begin + (int)(local / per_seg), tt = (int)((local % per_seg) / cs);
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
    const double tot = block_sum(row_min_partial(it.A.D + (int64_t)s * P, t == 0 ? (const real*)nullptr : it.M, P), red);
    if (threadIdx.x == 0) it.area[s] = tot;
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
