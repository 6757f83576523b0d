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
// Phases:
//   1  seeds: exact dot products cov(0, x) for every column (top row) and
//      cov(r, 0) for every row (left edge), in the working precision, from
//      series values held as hi + lo pairs about a tile reference and centred
//      locally before they are multiplied (covariance is shift-invariant)
//   2  rows r = 0 .. R-1: centred recurrence along diagonals
//        cov(r, x) = cov(r-1, x-1) + df_i dg_j + df_j dg_i
//      thread t owns the V columns tV .. tV+V-1.  The covariance is carried as
//      hi + lo: the updates of the last few rows accumulate in the small term lo,
//      which is folded into hi every FOLD rows, so hi is rounded FOLD times less
//      often than a plain running sum.  rho = (hi + lo) * a_i * a_j, and rho = 1
//      exactly where the row and column subsequences coincide (i == j).  Column
//      maxima (allP_BA, eq. 10) stay in registers; the row maxima over each
//      position's R-column window (allP_AB, eq. 11) come from van Herk /
//      Gil-Werman style prefix/suffix maxima over V-column chunks plus the maxima
//      of the whole chunks in between; one barrier per row
//   3  per position, the k-th largest of the 2R values of P_ABBA (eqs. 12-13)
//      by bisection on order-preserving integer keys; D = sqrt(2 ell max(0, 1-rho*))
#pragma once
#include <cstdint>
#include <cfloat>

#include "keys.cuh"

namespace pastila {

constexpr int FOLD = 8;  // rows between folds of the small covariance term

template <typename real> struct RealLimits;
template <> struct RealLimits<float> {
    __host__ __device__ static constexpr float lowest() { return -FLT_MAX; }
};
template <> struct RealLimits<double> {
    __host__ __device__ static constexpr double lowest() { return -DBL_MAX; }
};

template <typename real>
struct ProfileArgs {
    const double* T;     // n values (FP64)
    const double* mu;    // C window means (FP64)
    const real* a;       // C inverse norms (0 = flat window)
    const real* df;      // C
    const real* dg;      // C
    int64_t n, C, P;
    int m, ell, k, R, S;
    int W;               // positions per tile (multiple of 32)
    int ntiles;          // tiles per segment
    real* D;             // S x P output, row-major
    unsigned long long* dmax_key;  // KeyOf<double>::enc(max D), combined with atomicMax
};

// Shared-memory layout of one tile; identical on host and device.
struct TileGeom {
    int R, W, Wb, V, NT, NW, LA, RS, LP, ell, m;
    size_t off_AB, off_CB, off_PRE, off_CM, off_XCH, off_row, off_left, off_top, off_Tc, off_Tcl,
        off_Ts, off_Tsl, off_q, bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Smallest L >= need with L == 32 / V (mod 32): makes the chunk-swizzled layout
// (element e at (e mod V) * L + e / V) conflict-free both for a warp whose lanes
// stride by V and for a warp reading 32 consecutive elements from an aligned base.
__host__ __device__ inline int swz_len(int need, int V) {
    const int r = 32 / V;
    int L = need;
    while ((L & 31) != (r & 31)) ++L;
    return L;
}

template <typename real>
__host__ __device__ inline TileGeom tile_geom(int m, int ell, int W, int V) {
    typedef typename KeyOf<real>::type key_t;
    TileGeom g;
    g.m = m;
    g.ell = ell;
    g.R = m - ell + 1;
    g.W = W;
    g.Wb = W + g.R - 1;
    g.V = V;
    g.NT = ((g.Wb + V - 1) / V + 31) / 32 * 32;
    g.NW = g.NT / 32;
    g.LA = swz_len((W + V - 1) / V, V);
    g.RS = V * g.LA + 1;  // odd row stride: rows of one column fall in distinct banks
    g.LP = swz_len(g.NT, V);
    size_t o = 0;
    g.off_AB = o;   o = align16(o + sizeof(key_t) * (size_t)g.R * g.RS);
    g.off_CB = o;   o = align16(o + sizeof(key_t) * (size_t)(g.Wb + 32));
    g.off_PRE = o;  o = align16(o + sizeof(real) * 2 * (size_t)V * g.LP);
    g.off_CM = o;   o = align16(o + sizeof(real) * 2 * (size_t)(g.NT + 1));
    g.off_XCH = o;  o = align16(o + sizeof(real) * 4 * (size_t)g.NW);
    g.off_row = o;  o = align16(o + sizeof(real) * 5 * (size_t)g.R);
    g.off_left = o; o = align16(o + sizeof(real) * (size_t)g.R);
    g.off_top = o;  o = align16(o + sizeof(real) * (size_t)(g.NT * V));
    g.off_Tc = o;   o = align16(o + sizeof(real) * (size_t)(g.NT * V + ell + 64));
    g.off_Tcl = o;  o = align16(o + sizeof(real) * (size_t)(g.NT * V + ell + 64));
    g.off_Ts = o;   o = align16(o + sizeof(real) * (size_t)m);
    g.off_Tsl = o;  o = align16(o + sizeof(real) * (size_t)m);
    g.off_q = o;    o = align16(o + sizeof(real) * (size_t)(ell + 1));
    g.bytes = o;
    return g;
}

template <typename real>
__device__ __forceinline__ real rmax(real a, real b) { return a > b ? a : b; }

// Exact k-th largest key of the 2R values of P_ABBA at tile position p
// (AB column p and CB[p .. p+R-1]) by bisection over the key range.
template <typename key_t>
__device__ __forceinline__ key_t select_kth_bisect(const key_t* __restrict__ AB, int RS, int swp,
                                                   const key_t* __restrict__ CB, int p, int R,
                                                   int kk) {
    key_t lo = ~(key_t)0, hi = 0;
    for (int r = 0; r < R; ++r) {
        const key_t v = AB[r * RS + swp];
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    }
    for (int j = 0; j < R; ++j) {
        const key_t v = CB[p + j];
        lo = v < lo ? v : lo;
        hi = v > hi ? v : hi;
    }
    // invariant: count(>= lo) >= kk, count(>= hi + 1) < kk
    while (lo < hi) {
        const key_t mid = lo + (key_t)((hi - lo) >> 1) + 1;
        int c = 0;
        for (int r = 0; r < R; ++r) c += AB[r * RS + swp] >= mid;
        for (int j = 0; j < R; ++j) c += CB[p + j] >= mid;
        if (c >= kk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename real, int V>
__device__ __forceinline__ void profile_tile(const ProfileArgs<real>& A, const TileGeom& G, int s,
                                             int tt, unsigned char* __restrict__ sm) {
    typedef KeyOf<real> K;
    typedef typename K::type key_t;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NT = G.NT, NW = G.NW;
    const int R = A.R, ell = A.ell, m = A.m;
    const int64_t p0 = (int64_t)tt * A.W;
    const int Wp = (int)((A.P - p0) < (int64_t)A.W ? (A.P - p0) : (int64_t)A.W);
    const int Wb = Wp + R - 1;
    const int64_t i0 = (int64_t)s * m;

    key_t* AB = (key_t*)(sm + G.off_AB);
    key_t* CB = (key_t*)(sm + G.off_CB);
    real* PRE = (real*)(sm + G.off_PRE);
    real* CM = (real*)(sm + G.off_CM);
    real* XCH = (real*)(sm + G.off_XCH);  // [parity][hi/lo][warp]
    real* rdf = (real*)(sm + G.off_row);
    real* rdg = rdf + R;
    real* ra = rdg + R;
    real* rmu = ra + R;   // hi part of mu_i - refs
    real* rmul = rmu + R; // lo part
    real* lseed = (real*)(sm + G.off_left);
    real* top = (real*)(sm + G.off_top);
    real* Tc = (real*)(sm + G.off_Tc);    // T - refc as hi + lo pairs: exact to about
    real* Tcl = (real*)(sm + G.off_Tcl);  // twice the working precision
    real* Ts = (real*)(sm + G.off_Ts);
    real* Tsl = (real*)(sm + G.off_Tsl);
    real* q = (real*)(sm + G.off_q);

    // ---------------------------------------------------------------- stage
    const double refc = A.mu[p0];
    const double refs = A.mu[i0];
    const int nTc = Wb + ell - 1;
    for (int y = tid; y < NT * V + ell + 64; y += NT) {
        const double d = y < nTc ? A.T[p0 + y] - refc : 0.0;
        const real h = (real)d;
        Tc[y] = h;
        Tcl[y] = (real)(d - (double)h);
    }
    for (int u = tid; u < m; u += NT) {
        const double d = A.T[i0 + u] - refs;
        const real h = (real)d;
        Ts[u] = h;
        Tsl[u] = (real)(d - (double)h);
    }
    for (int r = tid; r < R; r += NT) {
        rdf[r] = A.df[i0 + r];
        rdg[r] = A.dg[i0 + r];
        ra[r] = A.a[i0 + r];
        const double d = A.mu[i0 + r] - refs;
        rmu[r] = (real)d;
        rmul[r] = (real)(d - (double)rmu[r]);
    }
    for (int t = tid; t < ell; t += NT) q[t] = (real)(A.T[i0 + t] - A.mu[i0]);
    __syncthreads();
    if (warp == 0) {  // sum of the rounded q, accumulated in FP64
        double acc = 0;
        for (int t = lane; t < ell; t += 32) acc += (double)q[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (lane == 0) q[ell] = (real)acc;
    }

    // ---------------------------------------------------------------- seeds
    // left edge: cov(r, 0) = sum_t (T[i+t] - mu_i) * (T[p0+t] - mu_p0); the row
    // values are centred term by term from their hi + lo parts, and mu of
    // column 0 is the reference of Tc
    for (int r = 1 + tid; r < R; r += NT) {
        const real mh = rmu[r], ml = rmul[r];
        real acc = 0;
        for (int t = 0; t < ell; ++t) acc += ((Ts[r + t] - mh) + (Tsl[r + t] - ml)) * (Tc[t] + Tcl[t]);
        lseed[r] = acc;
    }
    __syncthreads();
    // top row: cov(0, x) = sum_t q[t] * (T[x+t] - c) - (mu_x - c) * sum_t q[t] for any
    // constant c (the centred q sums to 0 up to rounding, and its rounded sum is
    // taken exactly).  c is the mean of each block's first column: the series
    // values of a block are centred once, from their hi + lo parts, as they enter
    // a sliding register window, so the products never carry the level of the
    // series, only its local deviations.  Lane-contiguous blocks of 9 columns
    // (odd stride: conflict-free sliding loads).
    {
        constexpr int J = 9;
        const int nblk = (NT * V + J - 1) / J;
        const real sq = q[ell];
        for (int b = tid; b < nblk; b += NT) {
            const int x0 = b * J;
            const double cb = x0 < Wb ? A.mu[p0 + x0] - refc : 0.0;
            const real cbh = (real)cb, cbl = (real)(cb - (double)cbh);
            real acc[J], win[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                acc[j] = 0;
                win[j] = (Tc[x0 + j] - cbh) + (Tcl[x0 + j] - cbl);
            }
            int t = 0;
            for (; t + J <= ell; t += J) {
#pragma unroll
                for (int u = 0; u < J; ++u) {
                    const real qt = q[t + u];
#pragma unroll
                    for (int j = 0; j < J; ++j) acc[j] += qt * win[(j + u) % J];
                    const int e = x0 + t + u + J;
                    win[u] = (Tc[e] - cbh) + (Tcl[e] - cbl);
                }
            }
            for (; t < ell; ++t) {
                const real qt = q[t];
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int e = x0 + t + j;
                    acc[j] += qt * ((Tc[e] - cbh) + (Tcl[e] - cbl));
                }
            }
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int x = x0 + j;
                if (x < Wb) {
                    const real dm = (real)(A.mu[p0 + x] - refc - cb);
                    top[x] = acc[j] - dm * sq;
                } else if (x < NT * V) {
                    top[x] = 0;
                }
            }
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- rows
    const int xb = tid * V;
    real hi[V], lo[V], cmx[V], cdf[V], cdg[V], ca[V];
    unsigned act = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int x = xb + v;
        if (x < Wb) {
            cdf[v] = A.df[p0 + x];
            cdg[v] = A.dg[p0 + x];
            ca[v] = A.a[p0 + x];
            act |= 1u << v;
        } else {
            cdf[v] = 0;
            cdg[v] = 0;
            ca[v] = 0;
        }
        hi[v] = top[x];
        lo[v] = 0;
        cmx[v] = RealLimits<real>::lowest();
    }
    const real NEG = RealLimits<real>::lowest();
    const int q0 = (R - 1) / V;  // chunk offset of the window end for i = 0
    // column of this thread's first cell on the main diagonal i == j at row r
    const int64_t xdiag0 = i0 - p0 - xb;

    for (int r = 0; r < R; ++r) {
        const int par = r & 1;
        real* PREp = PRE + par * V * G.LP;
        real* CMp = CM + par * (NT + 1);
        if (r > 0) {
            // cov(r-1, x-1) of this thread's first column: the neighbour lane's last
            // column, the previous warp's last column (lane 0), or, for tile column 0,
            // no predecessor at all: there cov(r, 0) is the exact left-edge seed
            real lhi = __shfl_up_sync(FULL, hi[V - 1], 1);
            real llo = __shfl_up_sync(FULL, lo[V - 1], 1);
            if (lane == 0 && warp > 0) {
                lhi = XCH[((par ^ 1) * 2 + 0) * NW + warp - 1];
                llo = XCH[((par ^ 1) * 2 + 1) * NW + warp - 1];
            }
            const real fr = rdf[r], gr = rdg[r];
#pragma unroll
            for (int v = V - 1; v >= 1; --v) {
                hi[v] = hi[v - 1];
                lo[v] = fr * cdg[v] + (cdf[v] * gr + lo[v - 1]);
            }
            if (tid == 0) {
                hi[0] = lseed[r];
                lo[0] = 0;
            } else {
                hi[0] = lhi;
                lo[0] = fr * cdg[0] + (cdf[0] * gr + llo);
            }
            if (r % FOLD == 0) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    hi[v] += lo[v];
                    lo[v] = 0;
                }
            }
        }
        if (lane == 31) {
            XCH[(par * 2 + 0) * NW + warp] = hi[V - 1];
            XCH[(par * 2 + 1) * NW + warp] = lo[V - 1];
        }
        real rho[V];
        const real ar = ra[r];
        if (ar != (real)0) {
#pragma unroll
            for (int v = 0; v < V; ++v) rho[v] = ((hi[v] + lo[v]) * ar) * ca[v];
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) rho[v] = ca[v] == (real)0 ? (real)1 : (real)0;
        }
        const int64_t xd = xdiag0 + r;  // i == j exactly: correlation 1 by definition
        if (xd >= 0 && xd < V) {
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (v == (int)xd) rho[v] = (real)1;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (!((act >> v) & 1u)) rho[v] = NEG;
            cmx[v] = rmax(cmx[v], rho[v]);
        }
        real pre[V], suf[V];
        pre[0] = rho[0];
#pragma unroll
        for (int v = 1; v < V; ++v) pre[v] = rmax(pre[v - 1], rho[v]);
        suf[V - 1] = rho[V - 1];
#pragma unroll
        for (int v = V - 2; v >= 0; --v) suf[v] = rmax(suf[v + 1], rho[v]);
#pragma unroll
        for (int v = 0; v < V; ++v) PREp[v * G.LP + tid] = pre[v];
        CMp[tid] = pre[V - 1];
        if (tid == 0) CMp[NT] = NEG;
        __syncthreads();
        // window maxima for the positions p = xb + i owned here
        if (xb < Wp) {
            // whole chunks strictly inside the window: tid+1 .. tid+q0-1 for small i,
            // one more (tid+q0) once the window end moves into chunk tid+q0+1
            real mid = NEG;
            for (int c = tid + 1; c < tid + q0; ++c) mid = rmax(mid, CMp[c]);
            const real mid1 = q0 >= 1 && tid + q0 <= NT ? rmax(mid, CMp[tid + q0]) : mid;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const int p = xb + i;
                if (p < Wp) {
                    real ab;
                    if (i + R - 1 < V) {  // window inside this chunk (R < V only)
                        ab = NEG;
#pragma unroll
                        for (int j = 0; j < V; ++j)
                            if (j >= i && j < i + R) ab = rmax(ab, rho[j]);
                    } else {
                        const int e = p + R - 1;
                        const int te = e / V;
                        ab = rmax(suf[i], te > tid + q0 ? mid1 : mid);
                        ab = rmax(ab, PREp[(e - te * V) * G.LP + te]);
                    }
                    AB[r * G.RS + i * G.LA + tid] = K::enc(ab);
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int x = xb + v;
        if (x < Wb) CB[x] = K::enc(cmx[v]);
    }
    __syncthreads();

    // ---------------------------------------------------------------- select
    const int kk = 2 * R > A.k ? A.k : 2 * R;
    const real two_ell = (real)(2 * ell);
    double tmax = 0.0;
    for (int p = tid; p < Wp; p += NT) {
        const int swp = (p % V) * G.LA + p / V;
        const key_t kb = select_kth_bisect<key_t>(AB, G.RS, swp, CB, p, R, kk);
        const real rs = K::dec(kb);
        real u = (real)1 - rs;
        u = u > (real)0 ? u : (real)0;
        const real d = sqrt(two_ell * u);
        A.D[(int64_t)s * A.P + p0 + p] = d;
        tmax = (double)d > tmax ? (double)d : tmax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(FULL, tmax, o);
        tmax = other > tmax ? other : tmax;
    }
    if (lane == 0) atomicMax(A.dmax_key, KeyOf<double>::enc(tmax));
}

// One CTA per (tile, segment): grid (ntiles, S).
template <typename real, int V>
__global__ void __launch_bounds__(512) profile_tiles_kernel(ProfileArgs<real> A, TileGeom G) {
    extern __shared__ __align__(16) unsigned char smem[];
    profile_tile<real, V>(A, G, blockIdx.y, blockIdx.x, smem);
}

}  // namespace pastila
