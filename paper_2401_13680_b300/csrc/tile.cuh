// The per-segment MPdist profile tile kernel (Section 4.1, eqs. 9-15).
//
// One CTA computes D_s(p) for one segment s and a tile of W consecutive profile
// positions p0 .. p0+Wp-1.  Everything is done in the correlation domain: the
// z-normalised distance d = sqrt(2 ell (1 - rho)) is a decreasing function of
// rho, so row/column minima of ED_matr (eqs. 10-11) are maxima of rho and the
// k-th smallest distance (eq. 13) is the k-th largest rho, mapped to a distance
// once at the end.
//
// Tile geometry (all indices tile-relative):
//   rows     r = 0 .. R-1   (ell-subsequence i = s*m + r of the segment)
//   columns  x = 0 .. Wb-1  (ell-subsequence j = p0 + x of T), Wb = Wp + R - 1
//   position p uses the R x R block rows 0..R-1, columns p .. p+R-1.
// Threads: NG row groups x NTc column threads.  Row group g walks rows
// g*Rg .. g*Rg+Rg-1; column thread t owns the V columns tV .. tV+V-1.  All
// groups step through their rows together, one barrier per step.
// Phases:
//   0  stage: bulk asynchronous copies (cp.async.bulk, completing on an
//      mbarrier) of the tile's series values and the segment's row statistics
//      into shared memory
//   1  seeds: exact dot products cov(g*Rg, x) for every column at the first row
//      of every row group, and cov(r, 0) for every row (left edge), in the
//      working precision, from series values held as hi + lo pairs and centred
//      locally before they are multiplied (covariance is shift-invariant)
//   2  rows: centred recurrence along diagonals
//        cov(r, x) = cov(r-1, x-1) + df_i dg_j + df_j dg_i
//      The covariance is carried as hi + lo: the updates of up to V rows
//      accumulate in the small term lo, folded into hi every V rows.  The V
//      registers of a thread hold consecutive columns; the diagonal shift from
//      row to row is a renaming of those registers inside an unrolled chunk of
//      V rows, plus one shuffle between lanes and a shared-memory exchange
//      between warps.  rho = (hi + lo) * a_i * a_j, and rho = 1 exactly where
//      the row and column subsequences coincide (i == j).  Column maxima
//      (allP_BA, eq. 10) stay in registers; the row maxima over each position's
//      R-column window (allP_AB, eq. 11) come from van Herk / Gil-Werman style
//      prefix/suffix maxima over V-column chunks plus the maxima of the whole
//      chunks in between.
//   3  per position, the k-th largest of the 2R values of P_ABBA (eqs. 12-13),
//      tracked from position to position: by groups of lanes on order-preserving
//      integer keys for R <= 288 (select_track), by one warp per run of positions
//      on values with incrementally updated counts beyond that (select_runs);
//      D = sqrt(2 ell max(0, 1-rho*))
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include <cfloat>

#include "keys.cuh"

namespace pastila {

// Bulk asynchronous copies from global to shared memory, completing on an
// mbarrier (the async copy engine moves the bytes; no thread issues loads).
// Both addresses must be 16-byte aligned and the size a multiple of 16.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes an initialised mbarrier visible to the async proxy
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity to complete, for at most `limit`
// SM clock cycles; false if it did not.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

template <typename real> struct RealLimits;
template <> struct RealLimits<float> {
    __host__ __device__ static constexpr float lowest() { return -FLT_MAX; }
    __host__ __device__ static constexpr float max() { return FLT_MAX; }
};
template <> struct RealLimits<double> {
    __host__ __device__ static constexpr double lowest() { return -DBL_MAX; }
    __host__ __device__ static constexpr double max() { return DBL_MAX; }
};

template <typename real>
struct ProfileArgs {
    const real* Th;      // n values of the series as hi + lo pairs (FP64: hi = value, lo = 0)
    const real* Tl;
    const real* muh;     // C window means as hi + lo pairs
    const real* mul;
    const real* a;       // C inverse norms (0 = flat window)
    const real* df;      // C
    const real* dg;      // C
    int64_t n, C, P;
    int m, ell, k, R, S;
    int W;               // positions per tile (multiple of 32)
    int ntiles;          // tiles per segment
    real* D;             // S x P output, row-major
    unsigned long long* dmax_key;  // KeyOf<double>::enc(max D), combined with atomicMax
    // streaming form (part != nullptr): D is not written; every CTA writes
    // part[(s - row_base) * ntiles + tile] = sum over its positions of
    // min(M_p, D_s(p)) (FP64, fixed order; M = nullptr: of D_s(p)), the greedy
    // areas without D
    const real* M;
    double* part;
    // with part: when pmx is not null, every CTA also writes the largest and the
    // smallest D_s(p) over its positions to pmx / pmn at the same index (the
    // sketch that bounds later greedy areas without recomputing the rows)
    real* pmx;
    real* pmn;
    // bounded waits: the staging wait gives up after spin_limit SM cycles and
    // then stores 1 to *err (host-visible); test_timeout is 0, and 1 only in
    // the test that makes the wait run out (a second wait, on the barrier's
    // next phase, which nothing completes)
    int* err;
    long long spin_limit;
    int test_timeout;
};

// Shared-memory layout and thread layout of one tile; identical on host and device.
struct TileGeom {
    int R, W, Wb, V, NTc, NWc, NG, Rg, NT, LA, RS, LP, ell, m;
    int GS;  // lanes per selection group (R <= 288: 4, 8, 16 or 32 with R <= 9 GS)
    // tiles of a thread-block cluster of CS CTAs (1, 2 or 4): CTA c computes rows
    // c Rh .. c Rh + Rh - 1 over every column of the tile and selects positions
    // c Wc .. c Wc + Wc - 1; AB holds all R rows of its own Wc positions (the
    // other CTAs write the rows they compute into it through distributed shared
    // memory), CBp[c'] the partial column maxima of CTA c'
    int CS, Rh, Wc;
    int RSt;  // stride of the five row-statistic arrays (room for a 16-byte-aligned copy of R values)
    size_t off_AB, off_CB, off_PRE, off_CM, off_LV, off_XCH, off_row, off_left, off_top, off_Tc, off_Tcl,
        off_Ts, off_Tsl, off_q, off_CBp, bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// NG_want row groups are asked for; the geometry uses Rg = ceil(R / NG_want)
// rows per group and as many groups as that needs.
template <typename real>
__host__ __device__ inline TileGeom tile_geom(int m, int ell, int W, int V, int NG_want, int CS = 1) {
    typedef typename KeyOf<real>::type key_t;
    TileGeom g;
    g.m = m;
    g.ell = ell;
    g.R = m - ell + 1;
    g.W = W;
    g.Wb = W + g.R - 1;
    g.V = V;
    g.NTc = ((g.Wb + V - 1) / V + 31) / 32 * 32;
    g.NWc = g.NTc / 32;
    g.CS = CS;
    g.Rh = (g.R + CS - 1) / CS;
    g.Wc = W / CS;
    g.Rg = (g.Rh + NG_want - 1) / NG_want;
    g.NG = (g.Rh + g.Rg - 1) / g.Rg;
    g.NT = g.NG * g.NTc;
    // AB row: position p at (p mod V) * LA + p / V, so the V-strided writes of a
    // row (thread t writes tV + i) are consecutive; an odd row stride keeps the
    // column reads of the selection (one position, many rows) in distinct banks
    g.LA = (g.Wc + V - 1) / V;
    g.RS = (V * g.LA) | 1;
    g.LP = g.NTc + 1;  // chunk prefix maxima: [V][LP], thread t at t (+ chunk offset)
    g.GS = g.R <= 36 ? 4 : (g.R <= 72 ? 8 : (g.R <= 144 ? 16 : 32));  // the narrowest that fits 9 values per half
    const size_t NG = (size_t)g.NG;
    size_t o = 0;
    g.off_AB = o;   o = align16(o + sizeof(key_t) * (size_t)g.R * g.RS);
    g.off_CB = o;   o = align16(o + sizeof(key_t) * (size_t)(g.Wb + 32));
    g.off_PRE = o;  o = align16(o + sizeof(real) * NG * 2 * (size_t)V * g.LP);
    g.off_CM = o;   o = align16(o + sizeof(real) * NG * 2 * (size_t)(g.NTc + 1));
    g.off_LV = o;   o = align16(o + sizeof(real) * NG * 2 * 4 * (size_t)g.NTc);
    g.off_XCH = o;  o = align16(o + sizeof(real) * NG * 4 * (size_t)g.NWc);
    // staged copies start at a 16-byte boundary at or below the data (up to
    // 16 / sizeof(real) - 1 elements early) and cover whole 16-byte units
    const int AE = 16 / (int)sizeof(real);
    g.RSt = (g.R + 2 * AE + AE - 1) / AE * AE;
    g.off_row = o;  o = align16(o + sizeof(real) * 5 * (size_t)g.RSt);
    g.off_left = o; o = align16(o + sizeof(real) * (size_t)g.R);
    g.off_top = o;  o = align16(o + sizeof(real) * NG * (size_t)(g.NTc * V));
    g.off_Tc = o;   o = align16(o + sizeof(real) * (size_t)(g.NTc * V + ell + 64));
    g.off_Tcl = o;  o = align16(o + sizeof(real) * (size_t)(g.NTc * V + ell + 64));
    g.off_Ts = o;   o = align16(o + sizeof(real) * (size_t)(m + 2 * AE));
    g.off_Tsl = o;  o = align16(o + sizeof(real) * (size_t)(m + 2 * AE));
    g.off_q = o;    o = align16(o + sizeof(real) * NG * (size_t)(ell + 1));
    g.off_CBp = o;  o = align16(o + (CS > 1 ? sizeof(real) * (size_t)CS * (g.Wb + 32) : 0));
    g.bytes = o;
    return g;
}

template <typename real>
__device__ __forceinline__ real rmax(real a, real b) { return a > b ? a : b; }

// Reductions over the G lanes of a group (G = 4, 8, 16 or 32 consecutive lanes;
// every lane of the warp takes part, each group reduces its own values).
template <typename T>
__device__ __forceinline__ T grp_sum(T v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
    return v;
}
// whole-warp groups: one redux.sync instead of a shuffle tree (32-bit values)
__device__ __forceinline__ uint32_t grp_sum(uint32_t v, int G) {
    if (G == 32) return __reduce_add_sync(0xffffffffu, v);
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
    return v;
}
__device__ __forceinline__ uint32_t grp_min(uint32_t v, int G) {
    if (G == 32) return __reduce_min_sync(0xffffffffu, v);
    for (int o = G >> 1; o > 0; o >>= 1) {
        const uint32_t w = __shfl_xor_sync(0xffffffffu, v, o, G);
        v = w < v ? w : v;
    }
    return v;
}
__device__ __forceinline__ uint32_t grp_max(uint32_t v, int G) {
    if (G == 32) return __reduce_max_sync(0xffffffffu, v);
    for (int o = G >> 1; o > 0; o >>= 1) {
        const uint32_t w = __shfl_xor_sync(0xffffffffu, v, o, G);
        v = w > v ? w : v;
    }
    return v;
}
template <typename T>
__device__ __forceinline__ T grp_min(T v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) {
        const T w = __shfl_xor_sync(0xffffffffu, v, o, G);
        v = w < v ? w : v;
    }
    return v;
}
template <typename T>
__device__ __forceinline__ T grp_max(T v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) {
        const T w = __shfl_xor_sync(0xffffffffu, v, o, G);
        v = w > v ? w : v;
    }
    return v;
}

// The working-precision type whose order-preserving key type is key_t.
template <typename key_t> struct KeyReal;
template <> struct KeyReal<uint32_t> { typedef float type; };
template <> struct KeyReal<unsigned long long> { typedef double type; };

constexpr int SEL_CACHE = 9;  // keys of one position held per lane, per half (rows, window)

// k-th largest key (kk-th, 1-based) of P_ABBA for a run of consecutive tile
// positions, one run per group of G lanes; all groups of a warp step through
// their runs together (npos_warp steps; a group past its own run idles on the
// CTA's first position).  Lane
// gl of a group holds rows gl, gl+G, ... of AB column p and the window entries
// CB[p+gl], CB[p+gl+G], ... in registers.  Every position after the first of
// a run starts from the previous answer tau (consecutive positions share all
// but a few of their 2R values, so the rank of tau moves little): a pass counts
// the keys >= tau and > tau, which settles most positions; otherwise a second
// pass finds the nearest key on the side the answer lies, which settles the
// answer when its rank moved by one, and tau steps to that key and the
// counting repeats.  The first position of a run,
// and a position still open after three steps, is searched inside its bracket
// of keys: the pivot interpolates between the values of two bounds with known
// counts (#{>= L} >= kk > #{>= H}) at the rank kk, and once a bound's count is
// exactly kk (or kk - 1 at H) one min (max) pass gives the answer; a bisection
// over the keys finishes anything still open after six pivots.  Control flow
// is uniform across the warp: decisions are per-group selects, loops run while
// any group of the warp still works.
template <typename key_t, typename Out>
__device__ __forceinline__ void select_track(const key_t* __restrict__ AB, int RS, int LA, int V,
                                             const key_t* __restrict__ CB, int R, int kk, int p_begin,
                                             int npos, int npos_warp, int G, int gl, int pofs, Out out) {
    // AB column of tile position p: p - pofs in this CTA's AB
    // requires R <= G * SEL_CACHE: every value of a position sits in the registers of its group
    typedef KeyOf<typename KeyReal<key_t>::type> K;
    typedef typename KeyReal<key_t>::type real;
    const unsigned FULL = 0xffffffffu;
    const key_t KMAX = ~(key_t)0;
    const int nr = (R - gl + G - 1) / G;  // values per half held by this lane
    key_t tau = 0;
    for (int it = 0; it < npos_warp; ++it) {
        const bool valid = it < npos;
        // an idle group (past the end of its run) reads this CTA's first
        // position, pofs, and takes no part in the searches
        const int p = valid ? p_begin + it : pofs;
        key_t va[SEL_CACHE], vb[SEL_CACHE];
        {
            const key_t* col = AB + ((p - pofs) % V) * LA + (p - pofs) / V + (size_t)gl * RS;
            const key_t* win = CB + p + gl;
#pragma unroll
            for (int j = 0; j < SEL_CACHE; ++j) {
                const bool in = j < nr;
                va[j] = in ? col[(size_t)j * G * RS] : (key_t)0;
                vb[j] = in ? win[j * G] : (key_t)0;
            }
        }
        key_t lo = 0, hi = KMAX;
        bool done = !valid;
        if (it > 0) {
            for (int step = 0; step < 3; ++step) {
                // counts alone settle most positions (the rank of tau did not move)
                uint32_t c = 0;
#pragma unroll
                for (int j = 0; j < SEL_CACHE; ++j) {
                    if (j < nr) {
                        const key_t a = va[j], b = vb[j];
                        c += (a >= tau ? 1u : 0u) + (a > tau ? 65536u : 0u);
                        c += (b >= tau ? 1u : 0u) + (b > tau ? 65536u : 0u);
                    }
                }
                c = grp_sum(c, G);
                const int cge = (int)(c & 0xffffu), cgt = (int)(c >> 16);
                if (!done) done = cgt < kk && kk <= cge;
                if (__all_sync(FULL, done)) break;
                // otherwise the nearest key on the side the answer lies: below tau when
                // fewer than kk keys are >= tau, above it when kk or more are > tau;
                // distance d = tau - 1 - a (below) or a - tau - 1 (above), both as
                // (a ^ s) + base, and keys on the wrong side wrap to large values
                const bool down = cge < kk;
                const key_t s = down ? ~(key_t)0 : (key_t)0, base = down ? tau : ~tau;
                key_t x = KMAX;
#pragma unroll
                for (int j = 0; j < SEL_CACHE; ++j) {
                    if (j < nr) {
                        const key_t da = (va[j] ^ s) + base, db = (vb[j] ^ s) + base;
                        x = da < x ? da : x;
                        x = db < x ? db : x;
                    }
                }
                x = grp_min(x, G);
                if (!done) {
                    if (down) {
                        tau = tau - (key_t)1 - x;
                        hi = tau;
                        done = cge == kk - 1;  // exactly one key short: the next key down is the answer
                    } else {
                        tau = tau + (key_t)1 + x;
                        lo = tau;
                        done = cgt == kk;      // exactly kk keys above: the smallest of them
                    }
                }
                if (__all_sync(FULL, done)) break;
            }
        }
        // search inside [lo, hi] (the whole key range at a run's first position):
        // interpolation on the values between two counted bounds, then the exact
        // answer by one min/max pass once a bound's count is exactly kk (or kk - 1
        // just above it); a bisection over the keys finishes whatever is left
        const bool need = !done;
        if (__any_sync(FULL, need)) {
            key_t mn = KMAX, mx = 0;
            uint32_t cb = 0;  // #{>= lo} + 65536 * #{> hi}
#pragma unroll
            for (int j = 0; j < SEL_CACHE; ++j) {
                if (j < nr) {
                    const key_t a = va[j], b = vb[j];
                    if (a >= lo && a <= hi) { mn = a < mn ? a : mn; mx = a > mx ? a : mx; }
                    if (b >= lo && b <= hi) { mn = b < mn ? b : mn; mx = b > mx ? b : mx; }
                    cb += (a >= lo ? 1u : 0u) + (a > hi ? 65536u : 0u) + (b >= lo ? 1u : 0u) + (b > hi ? 65536u : 0u);
                }
            }
            mn = grp_min(mn, G);
            mx = grp_max(mx, G);
            cb = grp_sum(cb, G);
            // bracket [L, H): #{>= L} = cL >= kk > cH = #{>= H}
            key_t L = mn, H = mx + (key_t)1;
            int cL = (int)(cb & 0xffffu), cH = (int)(cb >> 16);
            auto open = [&]() { return need && cL != kk && cH != kk - 1 && H - L > (key_t)1; };
            for (int itr = 0; itr < 6 && __any_sync(FULL, open()); ++itr) {
                const bool act = open();
                const real fL = K::dec(L), fH = K::dec(H);
                const real f = ((real)(cL - kk) + (real)0.5) / (real)(cL - cH);
                key_t pv = K::enc(fL + (fH - fL) * f);
                if (!(pv > L && pv < H)) pv = L + (key_t)((H - L) >> 1);
                uint32_t c = 0;
#pragma unroll
                for (int j = 0; j < SEL_CACHE; ++j)
                    if (j < nr) c += (va[j] >= pv ? 1u : 0u) + (vb[j] >= pv ? 1u : 0u);
                c = grp_sum(c, G);
                if (act) {
                    if ((int)c >= kk) { L = pv; cL = (int)c; } else { H = pv; cH = (int)c; }
                }
            }
            // exactly kk keys >= L: the answer is the smallest of them; exactly
            // kk - 1 keys >= H: the largest key below H
            const bool by_min = need && cL == kk, by_max = need && !by_min && cH == kk - 1;
            if (__any_sync(FULL, by_min || by_max)) {
                key_t lo_ge = KMAX, hi_lt = 0;
#pragma unroll
                for (int j = 0; j < SEL_CACHE; ++j) {
                    if (j < nr) {
                        const key_t a = va[j], b = vb[j];
                        if (a >= L) lo_ge = a < lo_ge ? a : lo_ge;
                        if (b >= L) lo_ge = b < lo_ge ? b : lo_ge;
                        if (a < H) hi_lt = a > hi_lt ? a : hi_lt;
                        if (b < H) hi_lt = b > hi_lt ? b : hi_lt;
                    }
                }
                lo_ge = grp_min(lo_ge, G);
                hi_lt = grp_max(hi_lt, G);
                if (by_min) { L = lo_ge; H = lo_ge + (key_t)1; }
                if (by_max) { L = hi_lt; H = hi_lt + (key_t)1; }
            }
            key_t blo = need ? L : tau, bhi = need ? H - (key_t)1 : tau;
            while (__any_sync(FULL, blo < bhi)) {
                const key_t mid = blo + (key_t)((bhi - blo) >> 1) + 1;
                uint32_t c = 0;
#pragma unroll
                for (int j = 0; j < SEL_CACHE; ++j)
                    if (j < nr) c += (va[j] >= mid ? 1u : 0u) + (vb[j] >= mid ? 1u : 0u);
                c = grp_sum(c, G);
                if (blo < bhi) {
                    if ((int)c >= kk) blo = mid; else bhi = mid - 1;
                }
            }
            tau = blo;
        }
        if (valid && gl == 0) out(p, tau);
    }
}

// The bits of a value in a key-typed shared-memory slot (the warp selector reads
// the slots back as values).
template <typename real>
__device__ __forceinline__ typename KeyOf<real>::type as_key(real v);
template <>
__device__ __forceinline__ uint32_t as_key<float>(float v) { return __float_as_uint(v); }
template <>
__device__ __forceinline__ unsigned long long as_key<double>(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

// Whole-warp reductions of working-precision values.
__device__ __forceinline__ float warp_max(float v) {
    return KeyOf<float>::dec(__reduce_max_sync(0xffffffffu, KeyOf<float>::enc(v)));
}
__device__ __forceinline__ float warp_min(float v) {
    return KeyOf<float>::dec(__reduce_min_sync(0xffffffffu, KeyOf<float>::enc(v)));
}
__device__ __forceinline__ double warp_max(double v) { return grp_max(v, 32); }
__device__ __forceinline__ double warp_min(double v) { return grp_min(v, 32); }

constexpr int SEL_CAP = 12;  // AB values of a column held per lane in registers (R <= 384)

// kk-th largest (1-based) of the 2R values of P_ABBA (eqs. 12-13) for a run of
// consecutive tile positions p_begin .. p_begin + npos - 1, one run per warp.
// Position p's values are AB column p (the R row-window maxima, eq. 11) and the
// window CB[p .. p+R-1] (column maxima, eq. 10); lane l holds rows l, l+32, ...
//
// The answer tau is tracked along the run together with the counts
// cge = #{x >= tau} and cgt = #{x > tau}.  From one position to the next only a
// few row-window maxima change (a window maximum changes only when it leaves the
// window or a larger value enters) and the column window slides by one, so the
// counts are updated from the changed values alone; tau stays the answer while
// cgt < kk <= cge.  Otherwise a pass over all 2R values finds the counts and the
// nearest values below and above tau and moves tau to the neighbour, up to three
// times, then a bisection inside the bracket found so far finishes; the first
// position of a run is found by bisection over the range of its values.  The
// bisections run over the order-preserving integer keys of the values (their
// midpoints are keys) but compare values, so equal values (+0 and -0 included)
// always count together.  Control flow is uniform across the warp.
// out(p, tau) is called by one lane per position, for 32 positions at a time.
template <typename real, typename Out>
__device__ __forceinline__ void select_runs(const real* __restrict__ AB, int RS, int LA, int V,
                                            const real* __restrict__ CB, int R, int kk, int p_begin,
                                            int npos, int pofs, Out out) {
    typedef KeyOf<real> K;
    typedef typename K::type key_t;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nrw = (R + 31) >> 5;  // entries per lane and half (the last may be partly empty)
    const real NEG = RealLimits<real>::lowest();
    const real POS = -NEG;
    real cur[SEL_CAP];              // AB column of the current position, rows lane + 32 j
    real tau = 0, mine = 0;
    int cge = 0, cgt = 0;
    int p = 0, cp = 0, cprev = 0;   // position; AB offsets of its column and of the previous one

    // f(x) for every value of position p held by this lane: rows, then window
    auto each = [&](auto&& f) {
#pragma unroll
        for (int j = 0; j < SEL_CAP; ++j) {
            const int r = lane + 32 * j;
            if (j < nrw && r < R) {
                f(cur[j]);
                f(CB[p + r]);
            }
        }
        for (int j = SEL_CAP; j < nrw; ++j) {
            const int r = lane + 32 * j;
            if (r < R) {
                f(AB[(size_t)r * RS + cp]);
                f(CB[p + r]);
            }
        }
    };
    auto count = [&]() {
        uint32_t c = 0;
        each([&](real x) { c += (x >= tau ? 1u : 0u) + (x > tau ? 65536u : 0u); });
        c = __reduce_add_sync(FULL, c);
        cge = (int)(c & 0xffffu);
        cgt = (int)(c >> 16);
    };
    // largest key v in [lo, hi] with #{x >= value(v)} >= kk
    auto bisect = [&](key_t lo, key_t hi) {
        while (lo < hi) {
            const key_t mid = lo + (key_t)((hi - lo) >> 1) + (key_t)1;
            const real mv = K::dec(mid);
            uint32_t c = 0;
            each([&](real x) { c += x >= mv ? 1u : 0u; });
            c = __reduce_add_sync(FULL, c);
            if ((int)c >= kk) lo = mid; else hi = mid - (key_t)1;
        }
        return K::dec(lo);
    };
    auto range = [&](key_t* lo, key_t* hi) {
        real mn = POS, mx = NEG;
        each([&](real x) {
            mn = x < mn ? x : mn;
            mx = x > mx ? x : mx;
        });
        *lo = K::enc(warp_min(mn));
        *hi = K::enc(warp_max(mx));
    };
    // tau from its previous value (the rank test has failed); leaves exact counts
    auto retrack = [&]() {
        key_t lo, hi;
        bool lo_set = false, hi_set = false;
        for (int step = 0; step < 3; ++step) {
            uint32_t c = 0;
            real below = NEG, above = POS;
            each([&](real x) {
                c += (x >= tau ? 1u : 0u) + (x > tau ? 65536u : 0u);
                below = (x < tau && x > below) ? x : below;
                above = (x > tau && x < above) ? x : above;
            });
            c = __reduce_add_sync(FULL, c);
            cge = (int)(c & 0xffffu);
            cgt = (int)(c >> 16);
            if (cgt < kk && kk <= cge) return;
            if (cge < kk) {  // the answer lies below tau
                tau = warp_max(below);
                hi = K::enc(tau);
                hi_set = true;
                if (cge == kk - 1) {
                    count();
                    return;
                }
            } else {         // above tau
                tau = warp_min(above);
                lo = K::enc(tau);
                lo_set = true;
                if (cgt == kk) {
                    count();
                    return;
                }
            }
        }
        key_t rlo, rhi;
        range(&rlo, &rhi);
        tau = bisect(lo_set ? lo : rlo, hi_set ? hi : rhi);
        count();
    };

    for (int it = 0; it < npos; ++it) {
        p = p_begin + it;
        cprev = cp;
        cp = ((p - pofs) % V) * LA + (p - pofs) / V;
        if (it == 0) {
#pragma unroll
            for (int j = 0; j < SEL_CAP; ++j) {
                const int r = lane + 32 * j;
                cur[j] = (j < nrw && r < R) ? AB[(size_t)r * RS + cp] : NEG;
            }
            key_t lo, hi;
            range(&lo, &hi);
            tau = bisect(lo, hi);
            count();
        } else {
            // count changes of the values that changed: rows, then the window slide
            int d = 0;
#pragma unroll
            for (int j = 0; j < SEL_CAP; ++j) {
                const int r = lane + 32 * j;
                if (j < nrw && r < R) {
                    const real nv = AB[(size_t)r * RS + cp], ov = cur[j];
                    d += ((nv >= tau) - (ov >= tau)) + 65536 * ((nv > tau) - (ov > tau));
                    cur[j] = nv;
                }
            }
            for (int j = SEL_CAP; j < nrw; ++j) {
                const int r = lane + 32 * j;
                if (r < R) {
                    const real nv = AB[(size_t)r * RS + cp], ov = AB[(size_t)r * RS + cprev];
                    d += ((nv >= tau) - (ov >= tau)) + 65536 * ((nv > tau) - (ov > tau));
                }
            }
            if (lane == 0) {
                const real ov = CB[p - 1];
                d -= (ov >= tau) + 65536 * (ov > tau);
            } else if (lane == 1) {
                const real nv = CB[p + R - 1];
                d += (nv >= tau) + 65536 * (nv > tau);
            }
            d = __reduce_add_sync(FULL, d);
            const int dge = (int)(int16_t)(d & 0xffff);
            cge += dge;
            cgt += (d - dge) >> 16;
            if (!(cgt < kk && kk <= cge)) retrack();
        }
        // lane (it mod 32) keeps this position's answer; 32 positions are written at once
        if (lane == (it & 31)) mine = tau;
        if ((it & 31) == 31 || it == npos - 1) {
            const int base = it & ~31;
            if (base + lane <= it) out(p_begin + base + lane, mine);
        }
    }
}

template <typename real, int V>
__device__ __forceinline__ void profile_tile(const ProfileArgs<real>& A, const TileGeom& G, int s,
                                             int tt, unsigned char* __restrict__ sm, int row_base = 0) {
    typedef KeyOf<real> K;
    typedef typename K::type key_t;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31;
    // a CTA may have more threads than the tile's layout uses (a batched launch
    // sized for its largest item): threads past G.NT only stage data and select
    const int BD = blockDim.x;
    const bool worker = tid < G.NT;
    const int NTc = G.NTc, NWc = G.NWc;
    const int RS = G.RS, LA = G.LA, LP = G.LP, NG = G.NG;  // read once: hot loops use registers
    const int g = worker ? tid / NTc : 0, t = tid % NTc, wc = t >> 5;  // row group, column thread, warp in group
    const int R = A.R, ell = A.ell, m = A.m, Rg = G.Rg;
    // cluster tiles: this CTA's rows and positions (one CTA: all of them)
    const int CS = G.CS;
    const int crank = CS > 1 ? (int)cooperative_groups::this_cluster().block_rank() : 0;
    const int rbase = crank * G.Rh, rend = rbase + G.Rh < R ? rbase + G.Rh : R;
    const int Wc = G.Wc;
    const int r0 = rbase + g * Rg;
    const int64_t p0 = (int64_t)tt * A.W;
    const int Wp = (int)((A.P - p0) < (int64_t)A.W ? (A.P - p0) : (int64_t)A.W);
    const int Wb = Wp + R - 1;
    const int64_t i0 = (int64_t)s * m;

    // row-window maxima (eq. 11), [row][position], and column maxima (eq. 10): as
    // order-preserving keys for the grouped selector (R <= 288), as values for the
    // warp selector
    const bool keyed = R <= 32 * SEL_CACHE;
    key_t* AB = (key_t*)(sm + G.off_AB);
    key_t* CB = (key_t*)(sm + G.off_CB);
    real* PRE = (real*)(sm + G.off_PRE) + (size_t)g * 2 * V * LP;  // this group's [parity][V][LP]
    real* CM = (real*)(sm + G.off_CM) + (size_t)g * 2 * (NTc + 1);   // [parity][NTc + 1]
    real* LV = (real*)(sm + G.off_LV) + (size_t)g * 2 * 4 * NTc;     // [parity][k-1][NTc]: max of the 2^k chunk
                                                                      // maxima from a chunk on, within its warp
    real* XCH = (real*)(sm + G.off_XCH) + (size_t)g * 4 * NWc;       // [parity][hi/lo][warp]
    // segment data are staged from the 16-byte boundary at or below i0
    constexpr int AE = 16 / (int)sizeof(real);
    const int os = (int)(i0 % AE);
    real* rowb = (real*)(sm + G.off_row);
    const int RSt = G.RSt;
    real* rdf = rowb + os;
    real* rdg = rowb + RSt + os;
    real* ra = rowb + 2 * RSt + os;
    real* rmu = rowb + 3 * RSt + os;  // mu_i as hi + lo
    real* rmul = rowb + 4 * RSt + os;
    real* lseed = (real*)(sm + G.off_left);
    real* top = (real*)(sm + G.off_top);  // [group][NTc * V] seeds, later the groups' column maxima
    real* Tc = (real*)(sm + G.off_Tc);    // the window's T as hi + lo pairs: exact to
    real* Tcl = (real*)(sm + G.off_Tcl);  // about twice the working precision
    real* Tsb = (real*)(sm + G.off_Ts);   // the segment's T, the same way
    real* Tslb = (real*)(sm + G.off_Tsl);
    real* Ts = Tsb + os;
    real* Tsl = Tslb + os;
    real* q = (real*)(sm + G.off_q);      // [group][ell + 1] centred head of the group's first row

    // ---------------------------------------------------------------- stage
    // Bulk asynchronous copies of the window's and the segment's series pairs
    // and the segment's five row statistics, completing on one mbarrier.  Each
    // copy starts at a 16-byte boundary (the window's start p0 is a multiple of
    // the tile width; the segment's is rounded down by os elements) and covers
    // whole 16-byte units (the device arrays carry padding past their ends).
    // No FP64 arithmetic: the series and the means arrive as pairs.  The wait
    // is bounded: past the limit the tile stores an error flag for the host and
    // goes on with whatever the shared memory holds, so that every barrier of
    // the tile (and of its cluster) is still reached.
    __shared__ uint64_t stage_bar;
    const int nTc = Wb + ell - 1;
    {
        const int64_t is = i0 - os;
        const uint32_t bw = (uint32_t)(sizeof(real) * ((nTc + AE - 1) / AE * AE));
        const uint32_t bs = (uint32_t)(sizeof(real) * ((os + m + AE - 1) / AE * AE));
        const uint32_t br = (uint32_t)(sizeof(real) * ((os + R + AE - 1) / AE * AE));
        if (tid == 0) {
            mbar_init(&stage_bar, 1);
            mbar_init_fence();
            mbar_arrive_expect_tx(&stage_bar, 2 * bw + 2 * bs + 5 * br);
            bulk_copy_g2s(Tc, A.Th + p0, bw, &stage_bar);
            bulk_copy_g2s(Tcl, A.Tl + p0, bw, &stage_bar);
            bulk_copy_g2s(Tsb, A.Th + is, bs, &stage_bar);
            bulk_copy_g2s(Tslb, A.Tl + is, bs, &stage_bar);
            bulk_copy_g2s(rowb, A.df + is, br, &stage_bar);
            bulk_copy_g2s(rowb + RSt, A.dg + is, br, &stage_bar);
            bulk_copy_g2s(rowb + 2 * RSt, A.a + is, br, &stage_bar);
            bulk_copy_g2s(rowb + 3 * RSt, A.muh + is, br, &stage_bar);
            bulk_copy_g2s(rowb + 4 * RSt, A.mul + is, br, &stage_bar);
        }
        // meanwhile: zeros past the copied window (columns beyond the tile feed
        // only discarded seeds)
        const int wcopied = (int)(bw / sizeof(real));
        for (int y = wcopied + tid; y < NTc * V + ell + 64; y += BD) {
            Tc[y] = (real)0;
            Tcl[y] = (real)0;
        }
    }
    // this thread's column statistics for the rows phase, loaded now so that
    // their latency passes under the staging and the seeds (FP32 path; the FP64
    // path has no registers to spare and loads them after the seeds)
    const int xb = t * V;
    real cdf[V], cdg[V], ca[V];
    auto load_cols = [&]() {
        if constexpr (sizeof(real) == 4 && V == 4) {
            if (xb + V <= Wb) {  // p0 + xb is a multiple of 4 (W is a multiple of 32): one 16-byte load each
                const float4 f = *reinterpret_cast<const float4*>(A.df + p0 + xb);
                const float4 gq = *reinterpret_cast<const float4*>(A.dg + p0 + xb);
                const float4 aq = *reinterpret_cast<const float4*>(A.a + p0 + xb);
                cdf[0] = f.x;
                cdf[1] = f.y;
                cdf[2] = f.z;
                cdf[3] = f.w;
                cdg[0] = gq.x;
                cdg[1] = gq.y;
                cdg[2] = gq.z;
                cdg[3] = gq.w;
                ca[0] = aq.x;
                ca[1] = aq.y;
                ca[2] = aq.z;
                ca[3] = aq.w;
                return;
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int x = xb + v;
            const bool in = x < Wb;
            cdf[v] = in ? A.df[p0 + x] : (real)0;
            cdg[v] = in ? A.dg[p0 + x] : (real)0;
            ca[v] = in ? A.a[p0 + x] : (real)0;
        }
    };
    constexpr bool early_cols = sizeof(real) == 4;
    if (early_cols) load_cols();
    const real c0h = A.muh[p0], c0l = A.mul[p0];  // mean of column 0, for the left seeds
    __syncthreads();  // the barrier is initialised before anyone waits on it
    {
        bool ok = mbar_wait_bounded(&stage_bar, 0, A.spin_limit);
        if (ok && A.test_timeout) ok = mbar_wait_bounded(&stage_bar, 1, A.spin_limit);
        if (!ok) *(volatile int*)A.err = 1;
    }
    // the groups' centred heads q = T[ig + u] - mu_ig, ig = i0 + rbase + gg Rg
    for (int e = tid; e < NG * ell; e += BD) {
        const int gg = e / ell, u = e - gg * ell;
        const int rb = rbase + gg * Rg;
        q[gg * (ell + 1) + u] = (Ts[rb + u] - rmu[rb]) + (Tsl[rb + u] - rmul[rb]);
    }
    __syncthreads();
    if ((tid >> 5) < NG) {  // warp gg: sum of group gg's rounded q, in FP64
        const int gg = tid >> 5;
        double acc = 0;
        for (int u = lane; u < ell; u += 32) acc += (double)q[gg * (ell + 1) + u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0) q[gg * (ell + 1) + ell] = (real)acc;
    }

    // ---------------------------------------------------------------- seeds
    // left edge: cov(r, 0) = sum_t (T[i+t] - mu_i) * (T[p0+t] - mu_p0), both
    // factors centred term by term from their hi + lo parts
    {
        // SPLIT consecutive lanes per row, lane sp summing the terms sp, sp + SPLIT,
        // ... (consecutive lanes, consecutive words), then a fixed-order shuffle sum:
        // short dependent chains, every thread busy
        const int rfirst = rbase > 1 ? rbase : 1;
        const int nrow = rend - rfirst;
        int SPLIT = 1;  // from the tile's own thread count: the same sums in every launch
        while (SPLIT < 32 && nrow > 0 && nrow * SPLIT * 2 <= G.NT) SPLIT *= 2;
        for (int base = 0; base < nrow * SPLIT; base += BD) {
            const int idx = base + tid;
            const int r = rfirst + idx / SPLIT, sp = idx % SPLIT;
            real acc = 0;
            if (r < rend) {
                const real mh = rmu[r], ml = rmul[r];
                for (int u = sp; u < ell; u += SPLIT)
                    acc += ((Ts[r + u] - mh) + (Tsl[r + u] - ml)) * ((Tc[u] - c0h) + (Tcl[u] - c0l));
            }
            for (int o = SPLIT >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o, SPLIT);
            if (r < rend && sp == 0) lseed[r] = acc;
        }
    }
    __syncthreads();
    // first row of every group: cov(r0, x) = sum_t q[t] * (T[x+t] - c) - (mu_x - c) * sum_t q[t]
    // for any constant c (the centred q sums to 0 up to rounding, and its rounded
    // sum is taken exactly).  c is the mean of each block's first column: the
    // series values of a block are centred once, from their hi + lo parts and
    // those of c, as they enter a sliding register window, so the products
    // never carry the level of the series, only its local deviations.  Lane-contiguous blocks of
    // 9 columns (odd stride: conflict-free sliding loads).
    {
        constexpr int J = 9;
        const int nblk = (NTc * V + J - 1) / J;
        for (int b = tid; b < NG * nblk; b += BD) {
            const int gg = b / nblk;
            const int x0 = (b - gg * nblk) * J;
            const real* qg = q + gg * (ell + 1);
            // every mean of the block loaded together (FP32 path; the FP64 path has
            // no registers to spare and loads them where they are used)
            constexpr bool early = sizeof(real) == 4;
            real mxh[J], mxl[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const bool in = early && x0 + j < Wb;
                mxh[j] = in ? A.muh[p0 + x0 + j] : (real)0;
                mxl[j] = in ? A.mul[p0 + x0 + j] : (real)0;
            }
            const real cbh = x0 < Wb ? (early ? mxh[0] : A.muh[p0 + x0]) : (real)0;
            const real cbl = x0 < Wb ? (early ? mxl[0] : A.mul[p0 + x0]) : (real)0;
            real acc[J], win[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                acc[j] = 0;
                win[j] = (Tc[x0 + j] - cbh) + (Tcl[x0 + j] - cbl);
            }
            int u0 = 0;
            for (; u0 + J <= ell; u0 += J) {
#pragma unroll
                for (int u = 0; u < J; ++u) {
                    const real qt = qg[u0 + u];
#pragma unroll
                    for (int j = 0; j < J; ++j) acc[j] += qt * win[(j + u) % J];
                    const int e = x0 + u0 + u + J;
                    win[u] = (Tc[e] - cbh) + (Tcl[e] - cbl);
                }
            }
            for (; u0 < ell; ++u0) {
                const real qt = qg[u0];
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int e = x0 + u0 + j;
                    acc[j] += qt * ((Tc[e] - cbh) + (Tcl[e] - cbl));
                }
            }
            const real sq = qg[ell];
            real* topg = top + (size_t)gg * NTc * V;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int x = x0 + j;
                if (x < Wb) {
                    const real dm = ((early ? mxh[j] : A.muh[p0 + x]) - cbh) + ((early ? mxl[j] : A.mul[p0 + x]) - cbl);
                    topg[x] = acc[j] - dm * sq;
                } else if (x < NTc * V) {
                    topg[x] = 0;
                }
            }
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- rows
    if (!early_cols) load_cols();
    const real NEG = RealLimits<real>::lowest();
    real hi[V], lo[V], cmx[V];
    const bool partial_cols = xb + V > Wb;  // only the last column thread of a tile
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int x = xb + v;
        hi[v] = worker ? top[(size_t)g * NTc * V + x] : (real)0;
        lo[v] = 0;
        cmx[v] = NEG;
    }
    const int q0 = (R - 1) / V;       // chunk offset of the window end for i = 0
    const bool small_R = R - 1 < V;   // some windows end inside their own chunk
    const int xdiag0 = (int)(i0 - p0) - xb;  // column (relative to xb) where i == j at row 0
    const bool owns_positions = worker && xb < Wp;
    const bool full_positions = xb + V <= Wp;
    const int nrows = !worker || r0 >= rend ? 0 : (r0 + Rg <= rend ? Rg : rend - r0);
    // the AB rows of this thread's V positions: in this CTA or, for the partner's
    // positions, in the partner's shared memory (all V positions share an owner:
    // Wc is a multiple of V)
    key_t* ABo = AB;
    int tofs = 0;
    if (CS > 1) {
        const int owner = owns_positions ? xb / Wc : crank;  // xb < Wp <= CS Wc when it owns positions
        tofs = owner * (Wc / V);
        if (owner != crank) ABo = cooperative_groups::this_cluster().map_shared_rank(AB, owner);
        // the partner must be running before its shared memory is written
        cooperative_groups::this_cluster().sync();
    }

    for (int c0 = 0; c0 < Rg; c0 += V) {
#pragma unroll
        for (int jj = 0; jj < V; ++jj) {
            const int sidx = c0 + jj;          // row step within the group
            const int r = r0 + sidx;
            const bool active = sidx < nrows;  // uniform within the group
            const int par = sidx & 1;
            real* PREp = PRE + par * V * LP;
            real* CMp = CM + par * (NTc + 1);
            real* LVp = LV + par * 4 * NTc;
            // logical column v of this thread lives in register (v - jj) mod V
            real rho[V];
            real pre = NEG;  // this thread's chunk maximum
            if (active) {
                if (sidx > 0) {
                    const int Pout = (V - jj) % V;  // register of the previous row's last column
                    real lhi = __shfl_up_sync(FULL, hi[Pout], 1);
                    real llo = __shfl_up_sync(FULL, lo[Pout], 1);
                    if (lane == 0 && wc > 0) {
                        lhi = XCH[((par ^ 1) * 2 + 0) * NWc + wc - 1];
                        llo = XCH[((par ^ 1) * 2 + 1) * NWc + wc - 1];
                    }
                    const real fr = rdf[r], gr = rdg[r];
#pragma unroll
                    for (int v = 1; v < V; ++v) {
                        const int P = (v - jj + V) % V;
                        lo[P] = fr * cdg[v] + (cdf[v] * gr + lo[P]);
                    }
                    if (t == 0) {
                        hi[Pout] = lseed[r];
                        lo[Pout] = 0;
                    } else {
                        hi[Pout] = lhi;
                        lo[Pout] = fr * cdg[0] + (cdf[0] * gr + llo);
                    }
                }
                if (lane == 31) {
                    const int Plast = (V - 1 - jj + V) % V;
                    XCH[(par * 2 + 0) * NWc + wc] = hi[Plast];
                    XCH[(par * 2 + 1) * NWc + wc] = lo[Plast];
                }
                const real ar = ra[r];
                if (ar != (real)0) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int P = (v - jj + V) % V;
                        rho[v] = ((hi[P] + lo[P]) * ar) * ca[v];
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) rho[v] = ca[v] == (real)0 ? (real)1 : (real)0;
                }
                const unsigned xd = (unsigned)(xdiag0 + r);  // i == j: correlation 1 by definition
                if (xd < (unsigned)V) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (v == (int)xd) rho[v] = (real)1;
                }
                if (partial_cols) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (xb + v >= Wb) rho[v] = NEG;
                }
#pragma unroll
                for (int v = 0; v < V; ++v) cmx[v] = rmax(cmx[v], rho[v]);
                pre = rho[0];
                PREp[t] = pre;
#pragma unroll
                for (int v = 1; v < V; ++v) {
                    pre = rmax(pre, rho[v]);
                    PREp[v * LP + t] = pre;
                }
                CMp[t] = pre;
                if (t == 0) CMp[NTc] = NEG;
                if (!small_R && q0 >= 2) {  // sparse table of the chunk maxima within each warp
                    real d = pre;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // entries reaching past the warp's end are never read
                        d = rmax(d, __shfl_down_sync(FULL, d, 1 << k));
                        LVp[k * NTc + t] = d;
                    }
                }
            }
            __syncthreads();
            // maximum of the whole chunks t+1 .. t+q0-1 strictly inside the windows of
            // this thread's positions, from the sparse tables: two overlapping spans of
            // 2^k chunks for the part in each warp the range touches, two spans of 16
            // for every whole warp in between
            real mid = NEG;
            if (active && owns_positions && !small_R && q0 >= 2) {
                auto span = [&](int x, int y) {  // x <= y in one warp
                    const int k = 31 - __clz(y - x + 1);
                    const real* Lk = k == 0 ? CMp : LVp + (k > 4 ? 3 : k - 1) * NTc;
                    const int w = k > 4 ? 16 : 1 << k;
                    return rmax(Lk[x], Lk[y - w + 1]);
                };
                const int a = t + 1, z = t + q0 - 1;
                const int wa = a >> 5, wz = z >> 5;
                if (wa == wz) {
                    mid = span(a, z);
                } else {
                    mid = rmax(span(a, wa * 32 + 31), span(wz * 32, z));
                    for (int w = wa + 1; w < wz; ++w) mid = rmax(mid, rmax(LVp[3 * NTc + w * 32], LVp[3 * NTc + w * 32 + 16]));
                }
            }
            if (active && owns_positions) {
                real suf[V];
                suf[V - 1] = rho[V - 1];
#pragma unroll
                for (int v = V - 2; v >= 0; --v) suf[v] = rmax(suf[v + 1], rho[v]);
                key_t* ABr = ABo + (size_t)r * RS + (t - tofs);
                if (!small_R) {
                    // whole chunks strictly inside the window: t+1 .. t+q0-1 (mid) for small
                    // i, one more (t+q0) once the window end moves into chunk t+q0+1
                    const real mid1 = rmax(mid, CMp[t + q0]);
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        const int e = i + R - 1;        // window end, relative to xb
                        const int oi = e / V, si = e - oi * V;
                        const real ab = rmax(rmax(suf[i], oi > q0 ? mid1 : mid), PREp[si * LP + t + oi]);
                        if (full_positions || xb + i < Wp) ABr[i * LA] = keyed ? K::enc(ab) : as_key<real>(ab);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        real ab;
                        if (i + R - 1 < V) {  // window inside this chunk
                            ab = NEG;
#pragma unroll
                            for (int j = 0; j < V; ++j)
                                if (j >= i && j < i + R) ab = rmax(ab, rho[j]);
                        } else {
                            const int e = i + R - 1;
                            const int oi = e / V, si = e - oi * V;
                            ab = rmax(suf[i], PREp[si * LP + t + oi]);
                        }
                        if (full_positions || xb + i < Wp) ABr[i * LA] = keyed ? K::enc(ab) : as_key<real>(ab);
                    }
                }
            }
        }
        // fold the small covariance term into the large one every V rows
#pragma unroll
        for (int v = 0; v < V; ++v) {
            hi[v] += lo[v];
            lo[v] = 0;
        }
    }
    // column maxima over all row groups
    {
        real* cmg = top + (size_t)g * NTc * V;
        if (worker) {
#pragma unroll
            for (int v = 0; v < V; ++v) cmg[xb + v] = cmx[v];
        }
    }
    __syncthreads();
    if (CS == 1) {
        for (int x = tid; x < Wb; x += BD) {
            real mx = top[x];
            for (int gg = 1; gg < NG; ++gg) mx = rmax(mx, top[(size_t)gg * NTc * V + x]);
            CB[x] = keyed ? K::enc(mx) : as_key<real>(mx);
        }
    } else {
        // this CTA's column maxima into slot crank of every CTA's CBp; after the
        // cluster barrier (which also completes every AB write into this CTA),
        // the maximum over the slots, in slot order
        real* CBp = (real*)(sm + G.off_CBp);
        const int slot = Wb + 32;
        for (int x = tid; x < Wb; x += BD) {
            real mx = top[x];
            for (int gg = 1; gg < NG; ++gg) mx = rmax(mx, top[(size_t)gg * NTc * V + x]);
            CBp[crank * slot + x] = mx;
        }
        for (int c = 0; c < CS; ++c) {
            if (c == crank) continue;
            real* CBq = cooperative_groups::this_cluster().map_shared_rank(CBp, c) + crank * slot;
            for (int x = tid; x < Wb; x += BD) CBq[x] = CBp[crank * slot + x];
        }
        cooperative_groups::this_cluster().sync();
        for (int x = tid; x < Wb; x += BD) {
            real mx = CBp[x];
            for (int c = 1; c < CS; ++c) mx = rmax(mx, CBp[c * slot + x]);
            CB[x] = keyed ? K::enc(mx) : as_key<real>(mx);
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- select
    const int kk = 2 * R > A.k ? A.k : 2 * R;
    const real two_ell = (real)(2 * ell);
    real tmax = 0;
    real tmin = RealLimits<real>::max();
    real* Drow = A.D + (int64_t)(s - row_base) * A.P + p0;  // row s - row_base of the output
    const bool streaming = A.part != nullptr;
    double sacc = 0.0;
    auto emit = [&](int p, real rs) {
        real u = (real)1 - rs;
        u = u > (real)0 ? u : (real)0;
        const real d = sqrt(two_ell * u);
        if (streaming) {
            const real mm = A.M ? A.M[p0 + p] : d;
            sacc += (double)(d < mm ? d : mm);
            tmin = d < tmin ? d : tmin;
        } else {
            Drow[p] = d;
        }
        tmax = d > tmax ? d : tmax;
    };
    // this CTA's positions: pofs .. pofs + Wn - 1 of the tile
    const int pofs = crank * Wc;
    const int Wn = Wp - pofs < 0 ? 0 : (Wp - pofs < Wc ? Wp - pofs : Wc);
    if (keyed) {
        // groups of GS lanes, each with a run of positions; a lane caches at most
        // SEL_CACHE values of each half
        const int GS = G.GS;
        const int ngroups = BD / GS;
        const int grp = tid / GS, gl = tid % GS;
        const int PW = (Wn + ngroups - 1) / ngroups;
        const int pb = grp * PW;
        const int npos = pb >= Wn ? 0 : (pb + PW <= Wn ? PW : Wn - pb);
        select_track<key_t>(AB, RS, LA, V, CB, R, kk, pofs + pb, npos, PW, GS, gl, pofs,
                            [&](int p, key_t kb) { emit(p, K::dec(kb)); });
    } else {
        // one run per warp; values beyond the register cache are read from shared memory
        const int nwarps = BD >> 5;
        const int PW = (Wn + nwarps - 1) / nwarps;
        const int pb = (tid >> 5) * PW;
        const int npos = pb >= Wn ? 0 : (pb + PW <= Wn ? PW : Wn - pb);
        select_runs<real>((const real*)AB, RS, LA, V, (const real*)CB, R, kk, pofs + pb, npos, pofs, emit);
    }
    const double wmax = warp_max(tmax);
    if (lane == 0) atomicMax(A.dmax_key, KeyOf<double>::enc(wmax));
    if (streaming) {  // this tile's area share: warps in order, then one store
        __shared__ double red[16];
        __shared__ real rmx[16], rmn[16];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(FULL, sacc, o);
        const real wmn = warp_min(tmin);
        if (lane == 0) {
            red[tid >> 5] = sacc;
            rmx[tid >> 5] = (real)wmax;
            rmn[tid >> 5] = wmn;
        }
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            real mx = rmx[0], mn = rmn[0];
            for (int w = 0; w < (BD >> 5); ++w) {
                tot += red[w];
                mx = rmx[w] > mx ? rmx[w] : mx;
                mn = rmn[w] < mn ? rmn[w] : mn;
            }
            const int64_t idx = ((int64_t)(s - row_base) * A.ntiles + tt) * CS + crank;
            A.part[idx] = tot;
            if (A.pmx) {
                A.pmx[idx] = mx;
                A.pmn[idx] = mn;
            }
        }
    }
}

// Streaming form over segments s_begin .. s_begin + gridDim.y - 1: grid (ntiles CS, segments).
template <typename real, int V>
__global__ void __launch_bounds__(512) stream_tiles_kernel(ProfileArgs<real> A, TileGeom G, int s_begin) {
    extern __shared__ __align__(16) unsigned char smem[];
    profile_tile<real, V>(A, G, s_begin + (int)blockIdx.y, (int)blockIdx.x / G.CS, smem, s_begin);
}

// The profile rows of a list of segments: CTA (tile, y) computes segment
// segs[y] into row y of A.D.  Grid: (ntiles CS, number of segments).
template <typename real, int V>
__global__ void __launch_bounds__(512) rows_tiles_kernel(ProfileArgs<real> A, TileGeom G,
                                                         const int32_t* __restrict__ segs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int s = segs[blockIdx.y];
    profile_tile<real, V>(A, G, s, (int)blockIdx.x / G.CS, smem, s - (int)blockIdx.y);
}

// One CTA (CS CTAs, a cluster) per (tile, segment): grid (ntiles CS, S).
template <typename real, int V>
__global__ void __launch_bounds__(512) profile_tiles_kernel(ProfileArgs<real> A, TileGeom G) {
    extern __shared__ __align__(16) unsigned char smem[];
    profile_tile<real, V>(A, G, blockIdx.y, (int)blockIdx.x / G.CS, smem);
}

}  // namespace pastila
