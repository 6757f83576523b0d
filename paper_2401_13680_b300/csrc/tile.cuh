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
//      tracked from position to position by one warp per run of positions, with
//      counts updated from the values that changed (select_warp);
//      D = sqrt(2 ell max(0, 1-rho*))
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include <cfloat>
#include <type_traits>

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

// Retires an mbarrier (its shared memory may then be used for anything else).
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Waits for the phase of the given parity to complete, for at most `limit`
// SM clock cycles; false if it did not.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// A cell of an FP32 tile whose row and column conditioning ratios (kappa,
// stats.cuh) multiply past this is recomputed by an exact dot product.  With
// the carry folded into hi every row, a float emulation of the recurrence on
// planted regimes and random walks (m = 64, 77; one group or groups of 10
// rows; seeds summed in blocks of 9 terms as below) keeps |d rho| below about
// 1.4e-7 kappa_i kappa_j -- most of it the rounding of the centred values
// themselves -- so 8 leaves about 1.1e-6, half of the 2e-6 the FP32 cells are
// held to.
constexpr float KAPPA_FLAG = 8.0f;

template <typename real> struct RealLimits;
template <> struct RealLimits<float> {
    __host__ __device__ static constexpr float lowest() { return -FLT_MAX; }
    __host__ __device__ static constexpr float max() { return FLT_MAX; }
};
template <> struct RealLimits<double> {
    __host__ __device__ static constexpr double lowest() { return -DBL_MAX; }
    __host__ __device__ static constexpr double max() { return DBL_MAX; }
};
template <> struct RealLimits<unsigned long long> {  // keys of FP64 values
    __host__ __device__ static constexpr unsigned long long lowest() { return 0ull; }
    __host__ __device__ static constexpr unsigned long long max() { return ~0ull; }
};

// Maxima and the selection compare FP32 values directly, and FP64 values by
// their order-preserving integer keys (B300 runs FP64 comparisons at a small
// fraction of the integer rate).  -0 is taken as +0 so that equal values have
// equal keys.
template <typename real> struct CmpOf { typedef real type; };
template <> struct CmpOf<double> { typedef unsigned long long type; };
__device__ __forceinline__ float to_cmp(float v) { return v; }
__device__ __forceinline__ unsigned long long to_cmp(double v) {
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    u = u == KeyOf<double>::TOP ? 0ull : u;
    return (u & KeyOf<double>::TOP) ? ~u : (u | KeyOf<double>::TOP);
}
__device__ __forceinline__ float cmp_value(float c) { return c; }
__device__ __forceinline__ double cmp_value(unsigned long long c) { return KeyOf<double>::dec(c); }
// the bits a shared-memory key slot holds for a compared quantity
__device__ __forceinline__ uint32_t cmp_bits(float c) { return __float_as_uint(c); }
__device__ __forceinline__ unsigned long long cmp_bits(unsigned long long c) { return c; }
// a key between kL and kH by interpolating the values at fraction f
__device__ __forceinline__ uint32_t interp_key(uint32_t kL, uint32_t kH, float f, uint32_t) {
    const float vL = KeyOf<float>::dec(kL), vH = KeyOf<float>::dec(kH);
    return KeyOf<float>::enc(vL + (vH - vL) * f);
}
__device__ __forceinline__ unsigned long long interp_key(unsigned long long kL, unsigned long long kH, float f,
                                                         unsigned long long) {
    const double vL = KeyOf<double>::dec(kL), vH = KeyOf<double>::dec(kH);
    return KeyOf<double>::enc(vL + (vH - vL) * (double)f);
}

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
    // FP32 tiles: C conditioning ratios of the windows (kappa_kernel); a cell
    // whose row and column ratios multiply past KAPPA_FLAG is recomputed
    // exactly.  nullptr: no check (FP64 tiles)
    const float* kappa;
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
    int R, W, Wb, V, NTc, NWc, NG, Rg, NT, LA, RS, ell, m;
    int GS;  // lanes per selection run (32: one warp per run of positions)
    // tiles of a thread-block cluster of CS CTAs (1, 2 or 4): CTA c computes rows
    // c Rh .. c Rh + Rh - 1 over every column of the tile and selects positions
    // c Wc .. c Wc + Wc - 1; AB holds all R rows of its own Wc positions (the
    // other CTAs write the rows they compute into it through distributed shared
    // memory), CBp[c'] the partial column maxima of CTA c'
    int CS, Rh, Wc;
    int RSt;  // stride of the five row-statistic arrays (room for a 16-byte-aligned copy of R values)
    size_t off_AB, off_CB, off_PRE, off_LV, off_XCH, off_rst, off_row, off_left, off_top, off_Tc, off_Tcl,
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
    g.GS = 32;  // lanes per selection run: one warp
    const size_t NG = (size_t)g.NG;
    size_t o = 0;
    g.off_AB = o;   o = align16(o + sizeof(key_t) * (size_t)g.R * g.RS);
    g.off_CB = o;   o = align16(o + sizeof(key_t) * (size_t)(g.Wb + 32));
    g.off_PRE = o;  o = align16(o + sizeof(real) * (NG * 2 * (size_t)(g.NTc * V) + 16));  // + reads past the last chunk
    g.off_LV = o;   o = align16(o + sizeof(real) * NG * 2 * 5 * (size_t)g.NTc);
    g.off_XCH = o;  o = align16(o + sizeof(real) * NG * 4 * (size_t)g.NWc);
    g.off_rst = o;  o = align16(o + sizeof(real) * 4 * (size_t)g.R);
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

// Whole-warp reductions of working-precision values.
__device__ __forceinline__ float warp_max(float v) {
    return KeyOf<float>::dec(__reduce_max_sync(0xffffffffu, KeyOf<float>::enc(v)));
}
__device__ __forceinline__ float warp_min(float v) {
    return KeyOf<float>::dec(__reduce_min_sync(0xffffffffu, KeyOf<float>::enc(v)));
}
__device__ __forceinline__ double warp_max(double v) { return grp_max(v, 32); }
__device__ __forceinline__ double warp_min(double v) { return grp_min(v, 32); }
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) { return grp_max(v, 32); }
__device__ __forceinline__ unsigned long long warp_min(unsigned long long v) { return grp_min(v, 32); }

constexpr int SEL_CAP = 12;  // most AB values of a column held per lane in registers (R <= 384)
constexpr int SEL_STEPS = 4;  // nearest-value steps before a position falls back to the bracketed search

// kk-th largest (1-based) of the 2R values of P_ABBA (eqs. 12-13) for a run of
// consecutive tile positions p_begin .. p_begin + npos - 1, one run per warp.
// Position p's values are AB column p (the R row-window maxima, eq. 11) and the
// window CB[p .. p+R-1] (column maxima, eq. 10); lane l holds rows l, l + 32, ...
// of the AB column in registers (the first SEL_CAP of them; rows beyond are read
// from shared memory) and reads its window entries CB[p + l + 32 j] where needed.
//
// The answer tau is carried along the run with the counts cge = #{x >= tau} and
// cgt = #{x > tau}; tau is the answer exactly when cgt < kk <= cge.  From one
// position to the next only a few row-window maxima change (a window maximum
// changes only when it leaves the window or a larger value enters) and the column
// window exchanges two values, so the counts are updated from the changed values
// alone.  When the rank test fails, the answer lies on one side of tau: one pass
// finds the nearest value on that side together with its multiplicity, which moves
// tau there with exact counts (for a move down, the values > new tau are those
// >= old tau); this repeats up to SEL_STEPS times.  The first position of a run,
// and a position still open after those steps, is found by a bracketed search:
// bounds L < H with known counts #{x >= L} >= kk > #{x >= H}, a pivot that
// interpolates their values at rank kk (bisection of the keys after eight pivots),
// and, once a bound's count is exactly kk (or kk - 1 at H), one nearest-value pass
// that gives the answer and its counts.  Every comparison is on values, so equal
// values (+0 and -0 included) count together; the order-preserving keys serve only
// the warp reductions and the midpoints.  Control flow is uniform across the warp.
// out(p, tau) is called by one lane per position, for 32 positions at a time.
// NJ: AB rows held per lane in registers (rows lane + 32 j, j < NJ); the caller
// picks the smallest NJ with 32 NJ >= R, or SEL_CAP (rows beyond are then read
// from shared memory).  NJV: rows j < NJV exist on every lane (R >= 32 NJV), so
// their tests compile away.  V: positions per AB row chunk (a power of two).
template <int NJ, int NJV, int V, typename real, typename Out>
__device__ __forceinline__ void select_warp(const real* __restrict__ AB, int RS, int LA,
                                            const real* __restrict__ CB, int R, int kk, int p_begin,
                                            int npos, int pofs, Out out) {
    typedef KeyOf<real> K;
    typedef typename K::type key_t;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nrw = (R + 31) >> 5;  // entries per lane and half (the last may be partly empty)
    const real NEG = RealLimits<real>::lowest();
    const real POS = RealLimits<real>::max();
    // this lane's rows lane + 32 j: offsets into AB and whether the row exists
    int roff[NJ];
    bool rin[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int r = lane + 32 * j;
        rin[j] = j < NJV || r < R;  // the caller guarantees R >= 32 NJV
        roff[j] = (rin[j] ? r : 0) * RS;
    }
    const real* CBl = CB + lane;    // window entry j of position p: CBl[p + 32 j]
    real cur[NJ];                   // AB column of the current position (NEG where no row)
    real tau = 0, mine = 0;
    int cge = 0, cgt = 0;
    int p = 0, cp = 0, cprev = 0;   // position; AB offsets of its column and of the previous one

    // f(x, valid) for every value of position p held by this lane: rows, then window
    auto each = [&](auto&& f) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            f(cur[j], rin[j]);
            f(rin[j] ? CBl[p + 32 * j] : NEG, rin[j]);
        }
        if constexpr (NJ == SEL_CAP) {  // below the cap, NJ rows per lane cover R
            for (int j = NJ; j < nrw; ++j) {
                const int r = lane + 32 * j;
                const bool in = r < R;
                f(in ? AB[r * RS + cp] : NEG, in);
                f(in ? CBl[p + 32 * j] : NEG, in);
            }
        }
    };
    auto count_ge = [&](real t) {  // t > NEG: absent entries never count
        int c = 0;
        each([&](real x, bool) { c += x >= t ? 1 : 0; });
        return (int)__reduce_add_sync(FULL, (unsigned)c);
    };
    // nearest value below t (max{x < t}) with its multiplicity over the position
    auto nearest_below = [&](real t, int* mult) {
        real best = NEG;
        int cnt = 0;
        each([&](real x, bool in) {
            const bool side = in && x < t;
            const bool better = side && x > best;
            cnt = better ? 1 : cnt + (side && x == best ? 1 : 0);
            best = better ? x : best;
        });
        const real w = warp_max(best);
        *mult = (int)__reduce_add_sync(FULL, (unsigned)(best == w ? cnt : 0));
        return w;
    };
    // nearest value above t (min{x > t}, or min{x >= t} with incl) with its multiplicity
    auto nearest_above = [&](real t, bool incl, int* mult) {
        real best = POS;
        int cnt = 0;
        each([&](real x, bool in) {
            const bool side = in && (x > t || (incl && x == t));
            const bool better = side && x < best;
            cnt = better ? 1 : cnt + (side && x == best ? 1 : 0);
            best = better ? x : best;
        });
        const real w = warp_min(best);
        *mult = (int)__reduce_add_sync(FULL, (unsigned)(best == w ? cnt : 0));
        return w;
    };
    // exact answer of position p by the bracketed search; sets tau, cge, cgt
    auto search = [&]() {
        real mn = POS, mx = NEG;
        each([&](real x, bool in) {
            mn = in && x < mn ? x : mn;
            mx = x > mx ? x : mx;
        });
        mn = warp_min(mn);
        mx = warp_max(mx);
        key_t kL = K::enc(mn), kH = K::enc(mx) + (key_t)1;
        int cL = 2 * R, cH = 0;  // #{x >= mn}, #{x >= the value after mx}
        for (int it = 0; it < 64; ++it) {
            int mult;
            if (cL == kk) {  // the answer is the smallest value >= L
                tau = nearest_above(K::dec(kL), true, &mult);
                cge = cL;
                cgt = cL - mult;
                return;
            }
            if (cH == kk - 1) {  // the answer is the largest value < H
                tau = nearest_below(K::dec(kH), &mult);
                cgt = cH;
                cge = cH + mult;
                return;
            }
            if (kH - kL <= (key_t)1) {  // only L itself lies in [L, H)
                tau = K::dec(kL);
                cge = cL;
                cgt = cH;
                return;
            }
            key_t kp = kL + (key_t)((kH - kL) >> 1);
            if (it < 8) {
                const float f = ((float)(cL - kk) + 0.5f) / (float)(cL - cH);
                const key_t ki = interp_key(kL, kH, f, key_t{});
                if (ki > kL && ki < kH) kp = ki;
            }
            const int c = count_ge(K::dec(kp));
            if (c >= kk) {
                kL = kp;
                cL = c;
            } else {
                kH = kp;
                cH = c;
            }
        }
        // not reached: past the eighth pivot the bracket halves every iteration
        tau = K::dec(kL);
        cge = cL;
        cgt = cH;
    };
    // contribution of one value to the packed counts (#{>= tau} + 65536 #{> tau})
    auto cnt2 = [&](real x) { return (x >= tau ? 1 : 0) + (x > tau ? 65536 : 0); };
    // packed counts of this lane's register-held AB values at tau (recounted
    // only when tau moves): a position's count change is then the new values'
    // counts less this
    auto held = [&]() {
        int c = 0;
#pragma unroll
        for (int j = 0; j < NJ; ++j) c += cnt2(cur[j]);
        return c;
    };
    // the column of the next position, loaded one position ahead so that the
    // loads overlap the current position's reductions
    real nxt[NJ];
    auto load_col = [&](int q, real* dst) {
        const int c = (q & (V - 1)) * LA + q / V;
#pragma unroll
        for (int j = 0; j < NJ; ++j) dst[j] = rin[j] ? AB[roff[j] + c] : NEG;
    };
    int ccur = 0;
    // the window slide: lane 0 adds the entering column maximum, lane 1 removes the leaving one
    const int wofs = lane == 0 ? R - 1 : -1;
    const int wsgn = lane == 0 ? 1 : (lane == 1 ? -1 : 0);

    // lane (it mod 32) keeps position it's answer; 32 positions are written at once
    auto keep = [&](int it) {
        if (lane == (it & 31)) mine = tau;
        if ((it & 31) == 31 || it == npos - 1) {
            const int base = it & ~31;
            if (base + lane <= it) out(p_begin + base + lane, mine);
        }
    };
    if (npos > 0) {  // the run's first position: the bracketed search
        p = p_begin;
        const int q = p - pofs;
        cp = (q & (V - 1)) * LA + q / V;
        load_col(q, cur);
        if (npos > 1) load_col(q + 1, nxt);
        search();
        ccur = held();
        keep(0);
    }
    for (int it = 1; it < npos; ++it) {
        p = p_begin + it;
        cprev = cp;
        const int q = p - pofs;
        cp = (q & (V - 1)) * LA + q / V;
        {
            // count changes of the values that changed: rows, then the window slide
            int nsum = 0;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                cur[j] = nxt[j];
                nsum += cnt2(cur[j]);
            }
            if (it + 1 < npos) load_col(q + 1, nxt);
            int d = nsum - ccur;
            ccur = nsum;
            if constexpr (NJ == SEL_CAP) {
                for (int j = NJ; j < nrw; ++j) {
                    const int r = lane + 32 * j;
                    if (r < R) d += cnt2(AB[r * RS + cp]) - cnt2(AB[r * RS + cprev]);
                }
            }
            d += wsgn * cnt2(CB[p + wofs]);
            d = (int)__reduce_add_sync(FULL, (unsigned)d);
            const int dge = (int)(int16_t)(d & 0xffff);
            cge += dge;
            cgt += (d - dge) >> 16;
            if (!(cgt < kk && kk <= cge)) {
                // the answer moved: step to the nearest value on its side, with exact counts
                for (int step = 0; step < SEL_STEPS && !(cgt < kk && kk <= cge); ++step) {
                    int mult;
                    if (cge < kk) {
                        tau = nearest_below(tau, &mult);
                        cgt = cge;
                        cge += mult;
                    } else {
                        tau = nearest_above(tau, false, &mult);
                        cge = cgt;
                        cgt -= mult;
                    }
                }
                if (!(cgt < kk && kk <= cge)) search();
                ccur = held();
            }
        }
        keep(it);
    }
}

template <typename real, int V>
__device__ __forceinline__ void profile_tile(const ProfileArgs<real>& A, const TileGeom& G, int s,
                                             int tt, unsigned char* __restrict__ sm, int row_base = 0) {
    typedef KeyOf<real> K;
    typedef typename K::type key_t;
    typedef typename CmpOf<real>::type cmp_t;  // what maxima and the selection compare
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31;
    // a CTA may have more threads than the tile's layout uses (a batched launch
    // sized for its largest item): threads past G.NT only stage data and select
    const int BD = blockDim.x;
    const bool worker = tid < G.NT;
    const int NTc = G.NTc, NWc = G.NWc;
    const int RS = G.RS, LA = G.LA, NG = G.NG;  // read once: hot loops use registers
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

    // row-window maxima (eq. 11), [row][position], and column maxima (eq. 10): FP32
    // tiles hold the values, FP64 tiles their order-preserving keys
    key_t* AB = (key_t*)(sm + G.off_AB);
    key_t* CB = (key_t*)(sm + G.off_CB);
    cmp_t* PRE = (cmp_t*)(sm + G.off_PRE) + (size_t)g * 2 * NTc * V;  // this group's [parity][column]: maxima
                                                                        // from the column's chunk start to it
    cmp_t* LV = (cmp_t*)(sm + G.off_LV) + (size_t)g * 2 * 5 * NTc;     // [parity][NTc][k]: max of the 2^k chunk
                                                                        // maxima from a chunk on, within its warp
    real* XCH = (real*)(sm + G.off_XCH) + (size_t)g * 4 * NWc;       // [warp][parity][hi, lo]
    real* rst = (real*)(sm + G.off_rst);                              // [row][df, dg, a, 0]
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
    // the largest conditioning ratio among this thread's columns (FP32 tiles
    // with the check)
    const float* kap = A.kappa;
    float kxm = 0.0f;
    if constexpr (sizeof(real) == 4) {
        if (kap) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (xb + v < Wb) kxm = fmaxf(kxm, kap[p0 + xb + v]);
        }
    }
    __shared__ unsigned kap_rmax;  // the rows' largest ratio, as float bits (all >= 0)
    if (tid == 0) kap_rmax = 0;
    const real c0h = A.muh[p0], c0l = A.mul[p0];  // mean of column 0, for the left seeds
    const float far_lim = 4.0f * rsqrtf((float)ell);
    __syncthreads();  // the barrier is initialised before anyone waits on it
    // staged: the copies of this thread's wait completed (if not, they may still
    // be in flight; the tile drains them before it ends)
    const bool staged = mbar_wait_bounded(&stage_bar, 0, A.spin_limit);
    {
        bool ok = staged;
        if (ok && A.test_timeout) ok = mbar_wait_bounded(&stage_bar, 1, A.spin_limit);
        if (!ok) *(volatile int*)A.err = 1;
    }
    if constexpr (sizeof(real) == 4) {
        if (kap) {
            float km = 0.0f;
            for (int r = rbase + tid; r < rend; r += BD) km = fmaxf(km, kap[i0 + r]);
            const unsigned b = __reduce_max_sync(FULL, __float_as_uint(km));
            if (lane == 0 && b) atomicMax(&kap_rmax, b);
        }
    }
    // the rows' statistics side by side (one 16-byte load per row step)
    bool flat_row = false;  // a row of this thread with a constant window (a_i = 0)
    for (int r = rbase + tid; r < rend; r += BD) {
        rst[4 * r + 0] = rdf[r];
        rst[4 * r + 1] = rdg[r];
        rst[4 * r + 2] = ra[r];
        rst[4 * r + 3] = (real)0;
        flat_row = flat_row || ra[r] == (real)0;
    }
    // the groups' centred heads q = T[ig + u] - mu_ig, ig = i0 + rbase + gg Rg
    for (int e = tid; e < NG * ell; e += BD) {
        const int gg = e / ell, u = e - gg * ell;
        const int rb = rbase + gg * Rg;
        q[gg * (ell + 1) + u] = (Ts[rb + u] - rmu[rb]) + (Tsl[rb + u] - rmul[rb]);
    }
    __syncthreads();
    // the sum of group gg's rounded q, in FP64, by warp gg of the caller's warps
    auto head_sums = [&](int w, int nw) {
        for (int gg = w; gg < NG; gg += nw) {
            double acc = 0;
            for (int u = lane; u < ell; u += 32) acc += (double)q[gg * (ell + 1) + u];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
            if (lane == 0) q[gg * (ell + 1) + ell] = (real)acc;
        }
    };

    // ---------------------------------------------------------------- seeds
    // left edge: cov(r, 0) = sum_t (T[i+t] - mu_i) * (T[p0+t] - mu_p0), both
    // factors centred term by term from their hi + lo parts; computed by the
    // threads lt = 0 .. nthr - 1 (a multiple of 32) of the caller's choice
    auto left_seeds = [&](int lt, int nthr) {
        // SPLIT consecutive lanes per row, lane sp summing the terms sp, sp + SPLIT,
        // ... (consecutive lanes, consecutive words), then a fixed-order shuffle sum:
        // short dependent chains
        const int rfirst = rbase > 1 ? rbase : 1;
        const int nrow = rend - rfirst;
        int SPLIT = 1;  // from the tile's own thread count: the same sums in every launch
        while (SPLIT < 32 && nrow > 0 && nrow * SPLIT * 2 <= G.NT) SPLIT *= 2;
        for (int base = 0; base < nrow * SPLIT; base += nthr) {
            const int idx = base + lt;
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
    };
    // first row of every group: cov(r0, x) = sum_t q[t] * (T[x+t] - c) - (mu_x - c) * sum_t q[t]
    // for any constant c (the centred q sums to 0 up to rounding, and its rounded
    // sum is taken exactly).  c is the mean of each block's first column: the
    // series values of a block are centred once, from their hi + lo parts and
    // those of c, as they enter a sliding register window, so the products
    // never carry the level of the series, only its local deviations.  Lane-contiguous blocks of
    // 9 columns (odd stride: conflict-free sliding loads).
    constexpr int J = 9;
    const int nblk = (NTc * V + J - 1) / J;
    // by threads gt = 0 .. nthr - 1 (nthr >= NG nblk: one block per thread); with
    // wait_sums, every one of them waits on barrier 1 for the groups' sums of q
    // (written by other warps, which arrive there) before the last step
    auto group_seeds = [&](int gt, int nthr, bool wait_sums) {
        const bool has = gt < NG * nblk;
        const int gg = has ? gt / nblk : 0;
        const int x0 = (gt - gg * nblk) * J;
        const real* qg = q + gg * (ell + 1);
        // every mean of the block loaded together (FP32 path; the FP64 path has
        // no registers to spare and loads them where they are used)
        constexpr bool early = sizeof(real) == 4;
        real mxh[J], mxl[J];
        real cbh = 0, cbl = 0;
        real acc[J];
#pragma unroll
        for (int j = 0; j < J; ++j) acc[j] = 0;
        if (has) {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const bool in = early && x0 + j < Wb;
                mxh[j] = in ? A.muh[p0 + x0 + j] : (real)0;
                mxl[j] = in ? A.mul[p0 + x0 + j] : (real)0;
            }
            cbh = x0 < Wb ? (early ? mxh[0] : A.muh[p0 + x0]) : (real)0;
            cbl = x0 < Wb ? (early ? mxl[0] : A.mul[p0 + x0]) : (real)0;
            real win[J];
#pragma unroll
            for (int j = 0; j < J; ++j) win[j] = (Tc[x0 + j] - cbh) + (Tcl[x0 + j] - cbl);
            int u0 = 0;
            for (; u0 + J <= ell; u0 += J) {
                // J terms summed apart, then added: the rounding of a seed grows with
                // J + ell / J terms rather than ell (an FP32 seed's error is carried,
                // scaled by the conditioning ratios, down its whole diagonal)
                real part[J];
#pragma unroll
                for (int j = 0; j < J; ++j) part[j] = 0;
#pragma unroll
                for (int u = 0; u < J; ++u) {
                    const real qt = qg[u0 + u];
#pragma unroll
                    for (int j = 0; j < J; ++j) part[j] += qt * win[(j + u) % J];
                    const int e = x0 + u0 + u + J;
                    win[u] = (Tc[e] - cbh) + (Tcl[e] - cbl);
                }
#pragma unroll
                for (int j = 0; j < J; ++j) acc[j] += part[j];
            }
            for (; u0 < ell; ++u0) {
                const real qt = qg[u0];
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int e = x0 + u0 + j;
                    acc[j] += qt * ((Tc[e] - cbh) + (Tcl[e] - cbl));
                }
            }
        }
        if (wait_sums) asm volatile("bar.sync 1, %0;" ::"r"(BD) : "memory");
        if (has) {
            const real sq = qg[ell];
            real* topg = top + (size_t)gg * NTc * V;
            unsigned far = 0;  // FP32: columns whose mean lies far from the block's centre
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int x = x0 + j;
                if (x < Wb) {
                    const real dm = ((early ? mxh[j] : A.muh[p0 + x]) - cbh) + ((early ? mxl[j] : A.mul[p0 + x]) - cbl);
                    topg[x] = acc[j] - dm * sq;
                    if constexpr (sizeof(real) == 4)
                        if (fabsf(dm) * A.a[p0 + x] > far_lim) far |= 1u << j;
                } else if (x < NTc * V) {
                    topg[x] = 0;
                }
            }
            // the products above carry |mu_x - c| besides the window's own deviations;
            // where that offset passes 4 / sqrt(ell) norms of the window (short windows,
            // level steps) their rounding would pass the recurrence's, so the seed is
            // taken again centred on the column's own mean
            while (far) {
                const int j = __ffs(far) - 1;
                far &= far - 1;
                const int x = x0 + j;
                const real mh = A.muh[p0 + x], ml = A.mul[p0 + x];
                real c0 = 0, c1 = 0;
                int u = 0;
                for (; u + 1 < ell; u += 2) {
                    c0 += qg[u] * ((Tc[x + u] - mh) + (Tcl[x + u] - ml));
                    c1 += qg[u + 1] * ((Tc[x + u + 1] - mh) + (Tcl[x + u + 1] - ml));
                }
                if (u < ell) c0 += qg[u] * ((Tc[x + u] - mh) + (Tcl[x + u] - ml));
                topg[x] = c0 + c1;
            }
        }
    };
    // The group seeds take one block of J columns per thread (fewer than half of
    // the CTA's threads); the left edge runs at the same time on the warps past
    // them, instead of before them on all threads.  Every sum is formed as it
    // would be by either arrangement.
    // The groups' sums of q come first, from the warps past the group seeds, which
    // then arrive on barrier 1; the group seeds wait there only before their last
    // step, which reads the sums.
    {
        const int tA = (NG * nblk + 31) / 32 * 32;
        if (tA + 32 <= BD) {  // the same for the whole CTA
            if (tid < tA) {
                group_seeds(tid, tA, true);
            } else {
                head_sums((tid - tA) >> 5, (BD - tA) >> 5);
                asm volatile("bar.arrive 1, %0;" ::"r"(BD) : "memory");
                left_seeds(tid - tA, BD - tA);
            }
        } else {
            head_sums(tid >> 5, BD >> 5);
            left_seeds(tid, BD);
            __syncthreads();
            group_seeds(tid, BD, false);
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- rows
    if (!early_cols) load_cols();
    // whether any cell of this thread can pass the conditioning flag (in most
    // tiles of most series none can, and the rows skip the check)
    const bool kap_check = kxm * __uint_as_float(kap_rmax) > KAPPA_FLAG;
    const real NEG = RealLimits<real>::lowest();
    const cmp_t NEGc = RealLimits<cmp_t>::lowest();
    real hi[V], lo[V];
    cmp_t cmx[V];
    const bool partial_cols = xb + V > Wb;  // only the last column thread of a tile
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int x = xb + v;
        hi[v] = worker ? top[(size_t)g * NTc * V + x] : (real)0;
        lo[v] = 0;
        cmx[v] = NEGc;
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

    // Loop-invariant parts of the row-window maxima of this thread's positions:
    // the maximum of the whole chunks t+1 .. t+q0-1 comes from the sparse tables
    // (two overlapping spans of 2^k chunks for the part in each warp the range
    // touches, two spans of 16 for every whole warp in between); so[] are those
    // table offsets.  The window of position xb + i ends at column xb + i + R - 1
    // (its prefix within its chunk is PRE[that column]) and covers chunk t + q0
    // entirely when i + rr >= V.
    const int rr = (R - 1) - q0 * V;
    int so[6] = {0, 0, 0, 0, 0, 0};  // so[4], so[5]: the first whole warp (else so[0] again)
    int wlo = 0, whi = -1;  // whole warps wlo .. whi between the spans
    const bool use_mid = owns_positions && !small_R && q0 >= 2;
    if (use_mid) {
        const int a = t + 1, z = t + q0 - 1;
        const int wa = a >> 5, wz = z >> 5;
        auto span = [&](int x, int y, int* o) {  // x <= y in one warp
            int k = 31 - __clz(y - x + 1);
            k = k > 4 ? 4 : k;
            o[0] = x * 5 + k;
            o[1] = (y - (1 << k) + 1) * 5 + k;
        };
        if (wa == wz) {
            span(a, z, so);
            so[2] = so[0];
            so[3] = so[1];
        } else {
            span(a, wa * 32 + 31, so);
            span(wz * 32, z, so + 2);
            wlo = wa + 1;
            whi = wz - 1;
        }
        so[4] = wlo <= whi ? wlo * 160 + 4 : so[0];
        so[5] = wlo <= whi ? wlo * 160 + 84 : so[0];
    }
    const int far0 = xb + R - 1;  // PRE column of the window end of position xb
    const bool far_vec = sizeof(real) == 4 && V == 4 && rr == 0;  // 16-byte aligned: xb and R - 1 multiples of 4
    // the common shape (every length of a sweep with ell = m / 2, m a multiple of
    // 8 and at most 520): windows of 3 to 66 chunks that end at a chunk boundary,
    // window ends read as one 16-byte load, at most one whole warp of chunks
    // between the two spans of the sparse tables.
    const bool common_rw = !small_R && far_vec && q0 >= 2 && q0 <= 65;  // at most one whole warp between the spans

    // A chunk of V row steps is FAST when the conditions that the row steps test
    // at every row are known for the whole tile: the common shape, all V rows of
    // every row group active, every owner's V positions in the tile and every
    // lane's columns wholly inside or wholly past the window (Wp a multiple of V:
    // the values past it are never read), no cell of the tile on the diagonal
    // i == j, and no row of the CTA with a constant window.  Fast chunks run a copy
    // of the row steps compiled with those conditions constant (their tests and
    // branches are a large share of a row step's instructions); the others run the
    // general copy.  The choice depends only on the tile and the chunk, so every
    // thread of the CTA (threads outside the layout included, which skip the row
    // work) runs the same copy and meets the same barriers.
    int nrows_min = Rg;  // rows of the shortest row group of the layout
    {
        const int last = rbase + (NG - 1) * Rg;
        const int nl = last >= rend ? 0 : (last + Rg <= rend ? Rg : rend - last);
        nrows_min = nl < Rg ? nl : Rg;
    }
    const int64_t dlo = i0 - p0 + rbase, dhi = i0 - p0 + rend - 1;  // diagonal columns of the CTA's rows
    bool tile_fast = common_rw && Wp % V == 0 && (dhi < 0 || dlo >= (int64_t)NTc * V);

    auto row_loop = [&](auto check_tag) {
    [[maybe_unused]] constexpr bool CHECK = decltype(check_tag)::value;
        key_t* ABr = ABo + (size_t)r0 * RS + (t - tofs);
        // mode 0: the general copy; 1: the fast copy; 2: the fast copy for a CTA
        // whose threads are all in the layout (every row step active)
        auto chunk = [&](int c0, auto mode_tag) {
        constexpr int MODE = decltype(mode_tag)::value;
        constexpr bool FAST = MODE > 0;
        const bool sR = FAST ? false : small_R;
        [[maybe_unused]] const bool fvec = FAST ? true : far_vec;
        const bool tables = FAST ? true : q0 >= 2;
        const bool mid_on = FAST ? true : use_mid;  // read where the thread owns positions
        const int rrc = FAST ? 0 : rr;
        const bool pcols = FAST ? false : partial_cols;
        const bool fullp = FAST ? true : full_positions;  // read where the thread owns positions
    #pragma unroll
            for (int jj = 0; jj < V; ++jj) {
                const int sidx = c0 + jj;          // row step within the group
                const int r = r0 + sidx;
                const bool active = MODE == 2 ? true : (FAST ? worker : sidx < nrows);  // uniform within the group
                const int par = sidx & 1;
                cmp_t* PREp = PRE + par * NTc * V;
                cmp_t* LVp = LV + par * 5 * NTc;
                // logical column v of this thread lives in register (v - jj) mod V
                cmp_t rc[V];
                if (active) {
                    real fr, gr, ar;
                    if constexpr (sizeof(real) == 4) {
                        const float4 q4 = *reinterpret_cast<const float4*>(rst + 4 * r);
                        fr = q4.x;
                        gr = q4.y;
                        ar = q4.z;
                    } else {
                        fr = rst[4 * r];
                        gr = rst[4 * r + 1];
                        ar = rst[4 * r + 2];
                    }
                    if (sidx > 0) {
                        const int Pout = (V - jj) % V;  // register of the previous row's last column
                        real lhi = __shfl_up_sync(FULL, hi[Pout], 1);
                        real llo = __shfl_up_sync(FULL, lo[Pout], 1);
                        if (lane == 0 && wc > 0) {
                            lhi = XCH[(wc - 1) * 4 + (par ^ 1) * 2 + 0];
                            llo = XCH[(wc - 1) * 4 + (par ^ 1) * 2 + 1];
                        }
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
                        if constexpr (sizeof(real) == 4) {
                            // fold the carry into hi every row (Dekker's fast two-sum): lo
                            // then holds one row's increments, not the diagonal's whole
                            // change, and its rounding shrinks with it
    #pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const real s = hi[v] + lo[v];
                                lo[v] = (hi[v] - s) + lo[v];
                                hi[v] = s;
                            }
                        }
                    }
                    if constexpr (sizeof(real) == 4) {
                        // ill-conditioned cells: the exact centred dot product instead of the
                        // recurrence (which then goes on from it along the diagonal)
                        if (CHECK && kap_check && sidx > 0) {
                            const float kr = kap[i0 + r];
                            if (kr * kxm > KAPPA_FLAG) {
                                const real mh = rmu[r], ml = rmul[r];
    #pragma unroll
                                for (int v = 0; v < V; ++v) {
                                    const int x = xb + v;
                                    if (x < Wb && kr * kap[p0 + x] > KAPPA_FLAG) {
                                        const real ch = A.muh[p0 + x], cl = A.mul[p0 + x];
                                        real c0 = 0, c1 = 0;
                                        int u = 0;
                                        for (; u + 1 < ell; u += 2) {
                                            c0 += ((Ts[r + u] - mh) + (Tsl[r + u] - ml)) * ((Tc[x + u] - ch) + (Tcl[x + u] - cl));
                                            c1 += ((Ts[r + u + 1] - mh) + (Tsl[r + u + 1] - ml)) *
                                                  ((Tc[x + u + 1] - ch) + (Tcl[x + u + 1] - cl));
                                        }
                                        if (u < ell) c0 += ((Ts[r + u] - mh) + (Tsl[r + u] - ml)) * ((Tc[x + u] - ch) + (Tcl[x + u] - cl));
                                        const int P = (v - jj + V) % V;
                                        hi[P] = c0 + c1;
                                        lo[P] = 0;
                                    }
                                }
                            }
                        }
                    }
                    if (lane == 31) {
                        const int Plast = (V - 1 - jj + V) % V;
                        XCH[wc * 4 + par * 2 + 0] = hi[Plast];
                        XCH[wc * 4 + par * 2 + 1] = lo[Plast];
                    }
                    {
                        real rho[V];
                        if (FAST || ar != (real)0) {
    #pragma unroll
                            for (int v = 0; v < V; ++v) {
                                const int P = (v - jj + V) % V;
                                // FP32: hi is the rounded sum of the pair (lo is below half its ulp)
                                rho[v] = ((sizeof(real) == 4 ? hi[P] : hi[P] + lo[P]) * ar) * ca[v];
                            }
                        } else {
    #pragma unroll
                            for (int v = 0; v < V; ++v) rho[v] = ca[v] == (real)0 ? (real)1 : (real)0;
                        }
                        const unsigned xd = (unsigned)(xdiag0 + r);  // i == j: correlation 1 by definition
                        if (!FAST && xd < (unsigned)V) {
    #pragma unroll
                            for (int v = 0; v < V; ++v)
                                if (v == (int)xd) rho[v] = (real)1;
                        }
    #pragma unroll
                        for (int v = 0; v < V; ++v) rc[v] = to_cmp(rho[v]);
                    }
                    if (pcols) {
    #pragma unroll
                        for (int v = 0; v < V; ++v)
                            if (xb + v >= Wb) rc[v] = NEGc;
                    }
    #pragma unroll
                    for (int v = 0; v < V; ++v) cmx[v] = rmax(cmx[v], rc[v]);
                    // prefix maxima within the chunk, stored by column
                    cmp_t pre[V];
                    pre[0] = rc[0];
    #pragma unroll
                    for (int v = 1; v < V; ++v) pre[v] = rmax(pre[v - 1], rc[v]);
                    if constexpr (sizeof(real) == 4 && V == 4) {
                        *reinterpret_cast<float4*>(PREp + xb) = make_float4(pre[0], pre[1], pre[2], pre[3]);
                    } else {
    #pragma unroll
                        for (int v = 0; v < V; ++v) PREp[xb + v] = pre[v];
                    }
                    if (!sR) {  // sparse table of the chunk maxima within each warp (level 0: the chunk maxima)
                        cmp_t d = pre[V - 1];
                        LVp[t * 5] = d;
                        if (tables) {
    #pragma unroll
                            for (int k = 0; k < 4; ++k) {  // entries reaching past the warp's end are never read
                                d = rmax(d, __shfl_down_sync(FULL, d, 1 << k));
                                LVp[t * 5 + k + 1] = d;
                            }
                        }
                    }
                }
                __syncthreads();
                if (active && owns_positions) {
                    cmp_t suf[V];
                    suf[V - 1] = rc[V - 1];
    #pragma unroll
                    for (int v = V - 2; v >= 0; --v) suf[v] = rmax(suf[v + 1], rc[v]);
                    if (!sR) {
                        // whole chunks strictly inside the windows: t+1 .. t+q0-1 (mid), and
                        // chunk t+q0 as well once the window end moves into chunk t+q0+1
                        cmp_t mid = NEGc;
                        if (mid_on) {
                            mid = rmax(rmax(LVp[so[0]], LVp[so[1]]), rmax(LVp[so[2]], LVp[so[3]]));
                            if (FAST) {
                                if (q0 > 33) mid = rmax(mid, rmax(LVp[so[4]], LVp[so[5]]));
                            } else {
                                for (int w = wlo; w <= whi; ++w)
                                    mid = rmax(mid, rmax(LVp[w * 160 + 4], LVp[w * 160 + 84]));
                            }
                        }
                        cmp_t far[V];
                        bool far_done = false;
                        if constexpr (sizeof(cmp_t) == 4 && V == 4) {
                            if (fvec) {
                                const float4 f4 = *reinterpret_cast<const float4*>(PREp + far0);
                                far[0] = f4.x;
                                far[1] = f4.y;
                                far[2] = f4.z;
                                far[3] = f4.w;
                                far_done = true;
                            }
                        }
                        if (!far_done) {
    #pragma unroll
                            for (int i = 0; i < V; ++i) far[i] = PREp[far0 + i];
                        }
                        const cmp_t mid1 = rrc > 0 ? rmax(mid, LVp[(t + q0) * 5]) : mid;
                        cmp_t ab[V];
    #pragma unroll
                        for (int i = 0; i < V; ++i) ab[i] = rmax(rmax(suf[i], i + rrc >= V ? mid1 : mid), far[i]);
                        if (fullp) {
    #pragma unroll
                            for (int i = 0; i < V; ++i) ABr[i * LA] = cmp_bits(ab[i]);
                        } else {
    #pragma unroll
                            for (int i = 0; i < V; ++i)
                                if (xb + i < Wp) ABr[i * LA] = cmp_bits(ab[i]);
                        }
                    } else {
    #pragma unroll
                        for (int i = 0; i < V; ++i) {
                            cmp_t ab;
                            if (i + R - 1 < V) {  // window inside this chunk
                                ab = NEGc;
    #pragma unroll
                                for (int j = 0; j < V; ++j)
                                    if (j >= i && j < i + R) ab = rmax(ab, rc[j]);
                            } else {
                                ab = rmax(suf[i], PREp[far0 + i]);
                            }
                            if (fullp || xb + i < Wp) ABr[i * LA] = cmp_bits(ab);
                        }
                    }
                }
                ABr += RS;
            }
            // FP64: fold the small covariance term into the large one every V rows
            // (FP32 folds it every row, keeping the remainder)
            if constexpr (sizeof(real) == 8) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    hi[v] += lo[v];
                    lo[v] = 0;
                }
            }
        };
        for (int c0 = 0; c0 < Rg; c0 += V) {
            if constexpr (sizeof(real) == 4 && V == 4) {
                if (tile_fast && c0 + V <= nrows_min) {  // the same for the whole CTA
                    if (BD == G.NT) chunk(c0, std::integral_constant<int, 2>{});
                    else chunk(c0, std::integral_constant<int, 1>{});
                } else {
                    chunk(c0, std::integral_constant<int, 0>{});
                }
            } else {
                chunk(c0, std::integral_constant<int, 0>{});
            }
        }
    };
    // The conditioning check is compiled into a second copy of the row loop,
    // taken only by tiles where some thread can meet the flag: in the others
    // the loop carries none of its code (a branch and an inner loop at every
    // row cost them about 7 % of their time even when never taken).
    if constexpr (sizeof(real) == 4) {
        tile_fast = tile_fast && !__syncthreads_or(flat_row);
        if (__syncthreads_or(kap_check)) row_loop(std::true_type{});
        else row_loop(std::false_type{});
    } else {
        row_loop(std::false_type{});
    }
    // column maxima over all row groups
    cmp_t* topc = (cmp_t*)top;  // the seeds are consumed: the groups' column maxima go here
    {
        cmp_t* cmg = topc + (size_t)g * NTc * V;
        if (worker) {
#pragma unroll
            for (int v = 0; v < V; ++v) cmg[xb + v] = cmx[v];
        }
    }
    __syncthreads();
    if (CS == 1) {
        for (int x = tid; x < Wb; x += BD) {
            cmp_t mx = topc[x];
            for (int gg = 1; gg < NG; ++gg) mx = rmax(mx, topc[(size_t)gg * NTc * V + x]);
            CB[x] = cmp_bits(mx);
        }
    } else {
        // this CTA's column maxima into slot crank of every CTA's CBp; after the
        // cluster barrier (which also completes every AB write into this CTA),
        // the maximum over the slots, in slot order
        cmp_t* CBp = (cmp_t*)(sm + G.off_CBp);
        const int slot = Wb + 32;
        for (int x = tid; x < Wb; x += BD) {
            cmp_t mx = topc[x];
            for (int gg = 1; gg < NG; ++gg) mx = rmax(mx, topc[(size_t)gg * NTc * V + x]);
            CBp[crank * slot + x] = mx;
        }
        for (int c = 0; c < CS; ++c) {
            if (c == crank) continue;
            cmp_t* CBq = cooperative_groups::this_cluster().map_shared_rank(CBp, c) + crank * slot;
            for (int x = tid; x < Wb; x += BD) CBq[x] = CBp[crank * slot + x];
        }
        cooperative_groups::this_cluster().sync();
        for (int x = tid; x < Wb; x += BD) {
            cmp_t mx = CBp[x];
            for (int c = 1; c < CS; ++c) mx = rmax(mx, CBp[c * slot + x]);
            CB[x] = cmp_bits(mx);
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
    auto emit = [&](int p, cmp_t rc_) {
        const real rs = cmp_value(rc_);
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
    {
        // one run per warp; values beyond the register cache are read from shared memory
        const int nwarps = BD >> 5;
        const int PW = (Wn + nwarps - 1) / nwarps;
        const int pb = (tid >> 5) * PW;
        const int npos = pb >= Wn ? 0 : (pb + PW <= Wn ? PW : Wn - pb);
        const cmp_t* ABv = (const cmp_t*)AB;
        const cmp_t* CBv = (const cmp_t*)CB;
        // NJ = ceil(R / 32) register rows per lane (R >= 32 (NJ - 1): all but the last on every lane)
        if (R <= 32) select_warp<1, 0, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else if (R <= 64) select_warp<2, 1, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else if (R <= 96) select_warp<3, 2, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else if (R <= 128) select_warp<4, 3, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else if (R <= 160) select_warp<5, 4, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else if (R <= 192) select_warp<6, 5, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else if (R <= 224) select_warp<7, 6, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else if (R <= 256) select_warp<8, 7, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else if (R <= 288) select_warp<9, 8, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
        else select_warp<SEL_CAP, 9, V, cmp_t>(ABv, RS, LA, CBv, R, kk, pofs + pb, npos, pofs, emit);
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
    // A staging wait that ran out may leave bulk copies (and their transaction
    // counts) in flight into this CTA's shared memory; they must not land after
    // the CTA has ended, in shared memory that another CTA may own by then.  Wait
    // for them again (bounded), then retire the barrier.  If that wait runs out
    // too, the barrier is left as it is (the error flag is already set).
    const bool drained = __syncthreads_and(staged) || mbar_wait_bounded(&stage_bar, 0, A.spin_limit);
    if (__syncthreads_and(drained) && tid == 0) mbar_inval(&stage_bar);
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
