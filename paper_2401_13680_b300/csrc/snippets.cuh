// Snippet search on the profile set D (S x P, row-major), Section 4.1 eqs. 16-17,
// the neighbour shares of eqs. 6-8, and the length criterion of eq. 18.
// All sums are FP64 with a fixed reduction order, so results are bit-identical
// from run to run.
#pragma once
#include <cstdint>

#include "keys.cuh"

namespace pastila {

constexpr int AREA_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// Exact widening of a binary32 value to binary64 (IEEE 754: every binary32
// value is a binary64 value) by moving its fields with integer operations:
// the sign stays, the exponent is rebiased by 1023 - 127 = 896, the 23
// fraction bits move to the top of the 52.  A subnormal input is first scaled
// by 2^24 in binary32 (exact, the result is normal) and rebiased by 896 - 24;
// zeros keep only their sign; infinities and NaNs get the all-ones exponent.
// The FP32 area sums use it instead of a conversion instruction, which on this
// GPU issues on the FP64 pipe, as slowly as the FP64 add itself.  The library is
// built without flush-to-zero, so the binary32 scaling keeps subnormal inputs
// (the exact-sum tests include them).
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float f) {
    const uint32_t u0 = __float_as_uint(f);
    const uint32_t e0 = u0 & 0x7F800000u;
    const bool sub = e0 == 0u;
    const uint32_t u = sub ? __float_as_uint(f * 16777216.0f) : u0;
    const uint32_t mag = u & 0x7FFFFFFFu;
    uint32_t hi = (mag >> 3) + ((sub ? 872u : 896u) << 20);
    if (e0 == 0x7F800000u) hi = 0x7FF00000u | ((mag & 0x007FFFFFu) >> 3);
    if (mag == 0u) hi = 0u;
    hi |= u0 & 0x80000000u;
    return __hiloint2double((int)hi, (int)(u << 29));
}

// This thread's share of sum_p min(M_p, row[p]) (M = nullptr: of row[p]) in a
// CTA of AREA_THREADS: positions tid, tid + AREA_THREADS, ... into four FP64
// accumulators in turn (four independent add chains), added pairwise at the
// end.  The areas stay FP64 sums (the precision plan keeps FP64 for them); on
// this GPU the FP64 adds, not the memory, set the kernel's speed, so the
// binary32 values are widened by integer operations (widen).  Every greedy area of the library goes through this one
// function, so the same row gives the same sum to the last bit in every path.
template <typename real>
__device__ __forceinline__ double row_min_partial(const real* __restrict__ row, const real* __restrict__ M,
                                                  int64_t P) {
    constexpr int64_t st = AREA_THREADS;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t p = threadIdx.x;
    if (M == nullptr) {
        for (; p + 3 * st < P; p += 4 * st) {
            a0 += widen(row[p]);
            a1 += widen(row[p + st]);
            a2 += widen(row[p + 2 * st]);
            a3 += widen(row[p + 3 * st]);
        }
        for (; p < P; p += st) a0 += widen(row[p]);
    } else {
        auto mn = [&](int64_t q) {
            const real d = row[q], mm = M[q];
            return widen(d < mm ? d : mm);
        };
        for (; p + 3 * st < P; p += 4 * st) {
            a0 += mn(p);
            a1 += mn(p + st);
            a2 += mn(p + 2 * st);
            a3 += mn(p + 3 * st);
        }
        for (; p < P; p += st) a0 += mn(p);
    }
    return (a0 + a1) + (a2 + a3);
}

// This thread's share of the error bound sum_p b(min(M_p, row[p])) (M = nullptr:
// +inf) of an FP32 area.  Every FP32 profile value x meets |x^2 - d64^2| <= c
// for the FP64 value d64 of the same cell (c = 2 ell |d rho| with the FP32
// path's accuracy |d rho| <= 2e-6, times 1.1 for the second-order terms), and
// min is 1-Lipschitz in each argument, so |min(M, x) - min(M64, d64)| <= b(x),
// b(x) = x - sqrt(x^2 - c) = c / (x + sqrt(x^2 - c)) for x^2 > c (the larger of
// the two sides), max(x, sqrt(x^2 + c) - x) otherwise.  In FP32: a bound, not
// an area; its own rounding, below 1 % for the sizes here, is covered by the
// caller's margin.
__device__ __forceinline__ float value_bound(float x, float c) {
    const float x2 = x * x;
    if (x2 > c) return c / (x + sqrtf(x2 - c));
    const float up = c / (sqrtf(x2 + c) + x);
    return x > up ? x : up;
}

template <typename real>
__device__ __forceinline__ float row_bound_partial(const real* __restrict__ row, const real* __restrict__ M,
                                                   int64_t P, float c) {
    constexpr int64_t st = AREA_THREADS;
    float a0 = 0.f, a1 = 0.f;
    int64_t p = threadIdx.x;
    auto term = [&](int64_t q) {
        float x = (float)row[q];
        if (M) {
            const float mm = (float)M[q];
            x = x < mm ? x : mm;
        }
        return value_bound(x, c);
    };
    for (; p + st < P; p += 2 * st) {
        a0 += term(p);
        a1 += term(p + st);
    }
    for (; p < P; p += st) a0 += term(p);
    return a0 + a1;
}

// area[s] = sum_p min(M_p, D_s(p)) for every segment s (M = +inf on the first
// step, so the area is the row sum).  One CTA per segment; chosen segments are
// skipped and get +inf.  Grid: (S).
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS)
area_kernel(const real* __restrict__ D, int S, int64_t P, const real* __restrict__ M,
            const int32_t* __restrict__ chosen, int nchosen, double* __restrict__ area) {
    __shared__ double red[AREA_THREADS / 32];
    const int s = blockIdx.x;
    bool skip = false;
    for (int t = 0; t < nchosen; ++t) skip |= chosen[t] == s;
    if (skip) {
        if (threadIdx.x == 0) area[s] = __longlong_as_double(0x7ff0000000000000ll);
        return;
    }
    const double tot = block_sum(row_min_partial(D + (int64_t)s * P, M, P), red);
    if (threadIdx.x == 0) area[s] = tot;
}

// The same per-row sum as area_kernel (same loop and reduction order, hence the
// same value to the last bit) for nrows contiguous rows: out[y] = sum_p
// min(M_p, rows[y][p]) (M = nullptr: the row sum).  Grid: (nrows).
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS)
row_area_kernel(const real* __restrict__ rows, int64_t P, const real* __restrict__ M, double* __restrict__ out) {
    __shared__ double red[AREA_THREADS / 32];
    const double tot = block_sum(row_min_partial(rows + (int64_t)blockIdx.x * P, M, P), red);
    if (threadIdx.x == 0) out[blockIdx.x] = tot;
}

// Block sketches of one streaming pass, for the segments of a chunk: over the
// tiles b TB .. (b+1) TB - 1 of segment s, the sum of the tiles' partial areas
// (A0, in tile order) and the largest and smallest profile value (X, N), from
// the per-CTA values of the pass; tot[s] = the block sums added in block order.
// Grid (segments), AREA_THREADS threads.
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS)
segment_sketch_kernel(const double* __restrict__ part, const real* __restrict__ pmx, const real* __restrict__ pmn,
                      int ntiles, int TB, int NB, double* __restrict__ A0, real* __restrict__ X, real* __restrict__ N,
                      double* __restrict__ tot) {
    const int s = blockIdx.x;
    const int64_t rt = (int64_t)s * ntiles, rb = (int64_t)s * NB;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) {
        const int t0 = b * TB, t1 = (b + 1) * TB < ntiles ? (b + 1) * TB : ntiles;
        double acc = 0.0;
        real mx = pmx[rt + t0], mn = pmn[rt + t0];
        for (int t = t0; t < t1; ++t) {
            acc += part[rt + t];
            mx = pmx[rt + t] > mx ? pmx[rt + t] : mx;
            mn = pmn[rt + t] < mn ? pmn[rt + t] : mn;
        }
        A0[rb + b] = acc;
        X[rb + b] = mx;
        N[rb + b] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < NB; ++b) t += A0[rb + b];
        tot[s] = t;
    }
}

// Lower bounds on the greedy areas sum_p min(M_p, D_s(p)) of step t (eq. 17)
// for segments whose rows are not at hand, block by block (blocks of L
// positions; Ms: the block's values of M sorted ascending, Mp: their running
// sums within the block):
//   D_s >= N_sb on the block:  sum min(M, D_s) >= sum min(M, N_sb)
//   D_s <= X_sb on the block:  sum min(M, D_s) = sum D_s - sum max(0, D_s - M)
//                                             >= A0_sb - sum max(0, X_sb - M)
//   block area Ab_sb known from step ts_s >= 1 (M only shrinks after it):
//                              sum min(M_t, D_s) >= Ab_sb - (MB_ts,b - MB_t,b)
// each also >= 0.  lb[s] = the sum over blocks of the largest of these, less
// rel times the magnitude of the sums involved (their FP64 rounding); taken
// segments get +inf.  Grid (S), AREA_THREADS threads.
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS)
stream_bounds_kernel(const double* __restrict__ A0, const double* __restrict__ Ab, const real* __restrict__ X,
                     const real* __restrict__ N, const int32_t* __restrict__ ts, const double* __restrict__ MB, int t,
                     const real* __restrict__ Ms, const double* __restrict__ Mp, int64_t P, int64_t L, int NB,
                     const unsigned char* __restrict__ taken, double rel, double* __restrict__ lb) {
    __shared__ double red[AREA_THREADS / 32], red2[AREA_THREADS / 32];
    const int s = blockIdx.x;
    if (taken[s]) {
        if (threadIdx.x == 0) lb[s] = __longlong_as_double(0x7ff0000000000000ll);
        return;
    }
    const int tss = ts[s];
    const int64_t rb = (int64_t)s * NB;
    double acc = 0.0, scale = 0.0;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) {
        const int64_t p0 = (int64_t)b * L;
        const int64_t Lb = p0 + L < P ? L : P - p0;
        const real* ms = Ms + p0;
        const double* mp = Mp + p0;
        auto below = [&](real v) {  // #{M < v} in the block
            int64_t lo = 0, hi = Lb;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (ms[mid] < v) lo = mid + 1; else hi = mid;
            }
            return lo;
        };
        const real n = N[rb + b], x = X[rb + b];
        const int64_t k1 = below(n), k2 = below(x);
        const double s1 = k1 ? mp[k1 - 1] : 0.0, s2 = k2 ? mp[k2 - 1] : 0.0;
        const double lbA = s1 + (double)n * (double)(Lb - k1);
        const double lbB = A0[rb + b] - ((double)x * (double)k2 - s2);
        double v = lbA > lbB ? lbA : lbB;
        if (tss >= 1) {
            const double lbD = Ab[rb + b] - (MB[(int64_t)tss * NB + b] - MB[(int64_t)t * NB + b]);
            v = lbD > v ? lbD : v;
        }
        acc += v > 0.0 ? v : 0.0;
        scale += A0[rb + b] + MB[(int64_t)t * NB + b] + (tss >= 1 ? MB[(int64_t)tss * NB + b] : 0.0);
    }
    const double tot = block_sum(acc, red);
    const double sc = block_sum(scale, red2);
    if (threadIdx.x == 0) lb[s] = tot - rel * sc;
}

// out[y][b] = sum over positions b*L .. min(P, (b+1)*L) - 1 of min(M_p, rows[y][p])
// (M = nullptr: of rows[y][p]).  Grid (NB, rows).
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS) row_blocks_kernel(const real* __restrict__ rows, int64_t P,
                                                                   const real* __restrict__ M, int64_t L, int NB,
                                                                   double* __restrict__ out) {
    __shared__ double red[AREA_THREADS / 32];
    const int b = blockIdx.x, y = blockIdx.y;
    const real* row = rows + (int64_t)y * P;
    const int64_t p0 = (int64_t)b * L, p1 = p0 + L < P ? p0 + L : P;
    double acc = 0.0;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += AREA_THREADS) {
        const real d = row[p];
        acc += widen(M && M[p] < d ? M[p] : d);
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) out[(int64_t)y * NB + b] = tot;
}

// out[b] = sum of M over positions b*L .. min(P, (b+1)*L) - 1.  Grid (NB).
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS) curve_blocks_kernel(const real* __restrict__ M, int64_t P, int64_t L,
                                                                     double* __restrict__ out) {
    __shared__ double red[AREA_THREADS / 32];
    const int64_t p0 = (int64_t)blockIdx.x * L, p1 = p0 + L < P ? p0 + L : P;
    double acc = 0.0;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += AREA_THREADS) acc += widen(M[p]);
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = tot;
}

// M <- row (first step) or min(M, row)
template <typename real>
__global__ void min_curve_kernel(const real* __restrict__ row, int64_t P, int first, real* __restrict__ M) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const real d = row[p];
    M[p] = first ? d : (d < M[p] ? d : M[p]);
}

// Nearest snippet per position (eq. 6) from the K chosen profiles stored as
// rows[t][p] (t in greedy order), lowest segment index on ties; counts[] must
// start at 0.
template <typename real>
__global__ void neighbors_rows_kernel(const real* __restrict__ rows, int64_t P, const int32_t* __restrict__ chosen,
                                      int K, int32_t* __restrict__ labels, unsigned long long* __restrict__ counts) {
    __shared__ unsigned int local[64];
    if (threadIdx.x < 64) local[threadIdx.x] = 0;
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) {
        int bt = 0;
        real bv = rows[p];
        for (int t = 1; t < K; ++t) {
            const real v = rows[(int64_t)t * P + p];
            if (v < bv || (v == bv && chosen[t] < chosen[bt])) {
                bv = v;
                bt = t;
            }
        }
        if (labels) labels[p] = chosen[bt];
        atomicAdd(&local[bt], 1u);
    }
    __syncthreads();
    if ((int)threadIdx.x < K && local[threadIdx.x])
        atomicAdd(&counts[threadIdx.x], (unsigned long long)local[threadIdx.x]);
}

// Greedy step: the unchosen segment with the smallest area (lowest index on
// ties) becomes chosen[t]; area_after[t] records its area.  One CTA of 1024.
__global__ void argmin_area_kernel(const double* __restrict__ area, int S, int32_t* __restrict__ chosen,
                                   double* __restrict__ area_after, int t) {
    __shared__ double bv[1024];
    __shared__ int bi[1024];
    double best = __longlong_as_double(0x7ff0000000000000ll);
    int bidx = 0x7fffffff;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double a = area[s];
        bool chosen_already = false;
        for (int u = 0; u < t; ++u) chosen_already |= chosen[u] == s;
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
        chosen[t] = bi[0];
        area_after[t] = bv[0];
    }
}

// M <- min(M, D_{chosen[t]}) (M = D_{chosen[0]} on the first step).
template <typename real>
__global__ void update_curve_kernel(const real* __restrict__ D, int64_t P, const int32_t* __restrict__ chosen,
                                    int t, real* __restrict__ M) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const real d = D[(int64_t)chosen[t] * P + p];
    if (t == 0) {
        M[p] = d;
    } else {
        const real mm = M[p];
        M[p] = d < mm ? d : mm;
    }
}

// Nearest snippet per position (eq. 6, argmin over the K chosen profiles, lowest
// segment index on ties) and per-snippet counts.  counts[] must start at 0.
template <typename real>
__global__ void neighbors_kernel(const real* __restrict__ D, int64_t P, const int32_t* __restrict__ chosen,
                                 int K, int32_t* __restrict__ labels,
                                 unsigned long long* __restrict__ counts) {
    __shared__ unsigned int local[64];
    if (threadIdx.x < 64) local[threadIdx.x] = 0;
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) {
        int bt = 0;
        real bv = D[(int64_t)chosen[0] * P + p];
        for (int t = 1; t < K; ++t) {
            const real v = D[(int64_t)chosen[t] * P + p];
            if (v < bv || (v == bv && chosen[t] < chosen[bt])) { bv = v; bt = t; }
        }
        if (labels) labels[p] = chosen[bt];
        atomicAdd(&local[bt], 1u);
    }
    __syncthreads();
    if ((int)threadIdx.x < K && local[threadIdx.x])
        atomicAdd(&counts[threadIdx.x], (unsigned long long)local[threadIdx.x]);
}

// frac (eq. 7) and the eq. 8 order (frac descending, segment index ascending).
// out_* are K records in eq. 8 order.  One thread.
__global__ void finalize_snippets_kernel(const int32_t* __restrict__ chosen, const double* __restrict__ area_after,
                                         const unsigned long long* __restrict__ counts, int K, int64_t P,
                                         int32_t* __restrict__ out_index, int32_t* __restrict__ out_rank,
                                         double* __restrict__ out_frac, double* __restrict__ out_area) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int order[64];
    for (int t = 0; t < K; ++t) order[t] = t;
    for (int i = 1; i < K; ++i) {
        const int x = order[i];
        int j = i - 1;
        while (j >= 0) {
            const int y = order[j];
            const bool before = counts[x] > counts[y] || (counts[x] == counts[y] && chosen[x] < chosen[y]);
            if (!before) break;
            order[j + 1] = y;
            --j;
        }
        order[j + 1] = x;
    }
    for (int i = 0; i < K; ++i) {
        const int t = order[i];
        out_index[i] = chosen[t];
        out_rank[i] = t;
        out_frac[i] = (double)counts[t] / (double)P;
        out_area[i] = area_after[t];
    }
}

// Numerator of eq. 18: partial[b] = sum over ordered pairs p != q of the chosen
// profiles of sum_{i in block b's range} |D_p(i) - D_q(i)|  (each unordered pair
// counted twice).  Grid: (nblocks); fixed ranges, fixed order.
template <typename real>
__global__ void __launch_bounds__(AREA_THREADS)
criterion_partial_kernel(const real* __restrict__ D, int64_t P, const int32_t* __restrict__ chosen, int K,
                         double* __restrict__ partial) {
    __shared__ double red[AREA_THREADS / 32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * AREA_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * AREA_THREADS + threadIdx.x; i < P; i += stride) {
        for (int a = 0; a < K; ++a) {
            const double x = (double)D[(int64_t)chosen[a] * P + i];
            for (int b = a + 1; b < K; ++b) {
                const double y = (double)D[(int64_t)chosen[b] * P + i];
                acc += fabs(x - y);
            }
        }
    }
    const double tot = block_sum(2.0 * acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// crit = sum(partial) / D_max (0 when D_max == 0).  One thread.
__global__ void criterion_final_kernel(const double* __restrict__ partial, int nb,
                                       const unsigned long long* __restrict__ dmax_key, double* __restrict__ crit) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double num = 0.0;
    for (int b = 0; b < nb; ++b) num += partial[b];
    const double den = KeyOf<double>::dec(*dmax_key);
    *crit = den > 0.0 ? num / den : 0.0;
}

// m_best = argmax crit (smallest m on ties).  One thread.
__global__ void select_best_kernel(const double* __restrict__ crit, const int32_t* __restrict__ ms, int n,
                                   int32_t* __restrict__ best_idx) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int b = 0;
    for (int i = 1; i < n; ++i)
        if (crit[i] > crit[b] || (crit[i] == crit[b] && ms[i] < ms[b])) b = i;
    *best_idx = b;
}

}  // namespace pastila
