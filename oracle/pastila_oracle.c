/*
 * Plain, slow FP64 CPU oracle of the paper's definitions (PaSTiLa, arXiv
 * 2401.13680).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark call it; the library never does.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * Every index here is 0-based.  T has n values; m is the segment length,
 * ell the inner subsequence length, R = m - ell + 1, P = n - m + 1 profile
 * positions, C = n - ell + 1 ell-subsequences, S = floor(n / m) segments.
 *
 * Parity status of each function (what pins it is in tests/test_oracle.py):
 *   ora_window_stats       pinned (numpy mean / std)
 *   ora_zdist              pinned (scipy zscore + norm; closed form 2*ell*(1-rho))
 *   ora_mpdist_pair        pinned (brute force with scipy cdist; ell = m reduces to
 *                          the z-normalised distance; k = 1 reduces to the min)
 *   ora_profiles_psf       pinned (equals ora_mpdist_pair cell by cell; invariants)
 *   ora_greedy             pinned (hand-computed cases; brute force of the rule)
 *   ora_neighbors          pinned (hand-computed cases; frac sums to 1)
 *   ora_criterion          pinned (hand-computed closed form; K = 1 gives 0)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Flat-window rule (the paper is silent): an ell-window whose centred sum of
 * squares is at most 1e-24 * ell * max(1, mu^2) has no z-normalisation.  Two
 * flat windows are at distance 0; a flat and a non-flat window at sqrt(2 ell),
 * the distance of correlation 0. */
#define ORA_FLAT_EPS 1e-24

static int ora_is_flat(double ss, double mu, int ell) {
    double s = mu * mu > 1.0 ? mu * mu : 1.0;
    return ss <= ORA_FLAT_EPS * (double)ell * s;
}

/* Mean and population standard deviation of every ell-window T[j .. j+ell),
 * j = 0 .. n-ell, by direct two-pass summation (definition of z-normalisation,
 * Section 4.1, the ED_norm distance of the technique the paper cites as [7]).
 * flat[j] = 1 marks a window with no z-normalisation. */
void ora_window_stats(const double* T, int64_t n, int ell, double* mu, double* sig,
                      int32_t* flat) {
    int64_t C = n - ell + 1;
    for (int64_t j = 0; j < C; ++j) {
        double s = 0.0;
        for (int t = 0; t < ell; ++t) s += T[j + t];
        double mj = s / ell;
        double ss = 0.0;
        for (int t = 0; t < ell; ++t) {
            double d = T[j + t] - mj;
            ss += d * d;
        }
        mu[j] = mj;
        sig[j] = sqrt(ss / ell);
        if (flat) flat[j] = ora_is_flat(ss, mj, ell);
    }
}

/* z-normalised Euclidean distance of two ell-windows, with explicit
 * z-vectors (x - mean) / std_pop (ED_norm in eq. 9). */
double ora_zdist(const double* x, const double* y, int ell) {
    double mx = 0.0, my = 0.0;
    for (int t = 0; t < ell; ++t) { mx += x[t]; my += y[t]; }
    mx /= ell;
    my /= ell;
    double sx = 0.0, sy = 0.0;
    for (int t = 0; t < ell; ++t) {
        sx += (x[t] - mx) * (x[t] - mx);
        sy += (y[t] - my) * (y[t] - my);
    }
    int fx = ora_is_flat(sx, mx, ell), fy = ora_is_flat(sy, my, ell);
    if (fx && fy) return 0.0;
    if (fx || fy) return sqrt(2.0 * ell);
    double dx = sqrt(sx / ell), dy = sqrt(sy / ell);
    double acc = 0.0;
    for (int t = 0; t < ell; ++t) {
        double d = (x[t] - mx) / dx - (y[t] - my) / dy;
        acc += d * d;
    }
    return sqrt(acc);
}

static int ora_cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* MPdist selection (eq. 13): sort P_ABBA ascending; if it holds more than k
 * values take the k-th smallest (1-based), else its largest value. */
static double ora_select(double* pabba, int len, int k) {
    qsort(pabba, (size_t)len, sizeof(double), ora_cmp_double);
    return len > k ? pabba[k - 1] : pabba[len - 1];
}

/* MPdist(A, B) of two length-m series from its pair definition: all
 * ell-subsequence distances E[r][c] between A and B, the matrix profile of A
 * against B (row minima, P_AB), of B against A (column minima, P_BA), their
 * concatenation and the eq. 13 selection. */
double ora_mpdist_pair(const double* A, const double* B, int m, int ell, int k) {
    int R = m - ell + 1;
    double* E = (double*)malloc(sizeof(double) * (size_t)R * R);
    double* pabba = (double*)malloc(sizeof(double) * 2 * (size_t)R);
    for (int r = 0; r < R; ++r)
        for (int c = 0; c < R; ++c) E[(size_t)r * R + c] = ora_zdist(A + r, B + c, ell);
    for (int r = 0; r < R; ++r) {
        double best = INFINITY;
        for (int c = 0; c < R; ++c) best = fmin(best, E[(size_t)r * R + c]);
        pabba[r] = best;
    }
    for (int c = 0; c < R; ++c) {
        double best = INFINITY;
        for (int r = 0; r < R; ++r) best = fmin(best, E[(size_t)r * R + c]);
        pabba[R + c] = best;
    }
    double v = ora_select(pabba, 2 * R, k);
    free(E);
    free(pabba);
    return v;
}

/* D_s(p) = MPdist(S_s, T[p .. p+m)) for the listed (segment, position) cells,
 * from the pair definition (eqs. 14-15). */
void ora_profile_cells(const double* T, int64_t n, int m, int ell, int k,
                       const int32_t* segs, const int64_t* pos, int64_t ncells, double* out) {
    (void)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < ncells; ++q)
        out[q] = ora_mpdist_pair(T + (int64_t)segs[q] * m, T + pos[q], m, ell, k);
}

/* Profiles D_s(p) for the listed segments and the positions p_lo .. p_hi-1,
 * following the PSF steps of Section 4.1 in order (only the columns those
 * positions need, j = p_lo .. p_hi-1+m-ell):
 *   eq. 9   ED_matr(r, j) = ED_norm(seg_{r,ell}, T_{j,ell}), r < R
 *   eq. 10  allP_BA(j)    = min_r ED_matr(r, j)
 *   eq. 11  allP_AB(r, p) = min_{p <= c <= p+m-ell} ED_matr(r, c)
 *   eq. 12  P_ABBA(p)     = {allP_AB(r, p)}_r  ++  {allP_BA(j)}_{p <= j <= p+m-ell}
 *   eq. 13  D_s(p)        = k-th smallest of P_ABBA(p), or its max if |P_ABBA| <= k
 * Output D is nsegs x (p_hi - p_lo) row-major. */
void ora_profiles_psf_range(const double* T, int64_t n, int m, int ell, int k,
                            const int32_t* segs, int nsegs, int64_t p_lo, int64_t p_hi, double* D) {
    (void)n;
    int R = m - ell + 1;
    int64_t np = p_hi - p_lo, nc = np + R - 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < nsegs; ++q) {
        const double* seg = T + (int64_t)segs[q] * m;
        double* ED = (double*)malloc(sizeof(double) * (size_t)R * (size_t)nc);
        double* pBA = (double*)malloc(sizeof(double) * (size_t)nc);
        double* pAB = (double*)malloc(sizeof(double) * (size_t)R * (size_t)np);
        double* pabba = (double*)malloc(sizeof(double) * 2 * (size_t)R);
        for (int r = 0; r < R; ++r)
            for (int64_t c = 0; c < nc; ++c) ED[(size_t)r * nc + c] = ora_zdist(seg + r, T + p_lo + c, ell);
        for (int64_t c = 0; c < nc; ++c) {
            double best = INFINITY;
            for (int r = 0; r < R; ++r) best = fmin(best, ED[(size_t)r * nc + c]);
            pBA[c] = best;
        }
        for (int r = 0; r < R; ++r)
            for (int64_t p = 0; p < np; ++p) {
                double best = INFINITY;
                for (int c = 0; c < R; ++c) best = fmin(best, ED[(size_t)r * nc + p + c]);
                pAB[(size_t)r * np + p] = best;
            }
        for (int64_t p = 0; p < np; ++p) {
            for (int r = 0; r < R; ++r) pabba[r] = pAB[(size_t)r * np + p];
            for (int c = 0; c < R; ++c) pabba[R + c] = pBA[p + c];
            D[(size_t)q * np + p] = ora_select(pabba, 2 * R, k);
        }
        free(ED);
        free(pBA);
        free(pAB);
        free(pabba);
    }
}

/* Full profiles of the listed segments: all P = n - m + 1 positions. */
void ora_profiles_psf(const double* T, int64_t n, int m, int ell, int k,
                      const int32_t* segs, int nsegs, double* D) {
    ora_profiles_psf_range(T, n, m, ell, k, segs, nsegs, 0, n - m + 1, D);
}

/* Greedy snippet search on ProfileArea (eqs. 16-17).  M starts at +inf; step t
 * picks, among segments not yet chosen, the s minimising
 * sum_p min(M_p, D_s(p)) over all P positions (lowest s on ties), then
 * M <- min(M, D_s).  area_after[t] is that minimum.  D is S x P row-major. */
void ora_greedy(const double* D, int S, int64_t P, int K, int32_t* chosen, double* area_after) {
    double* M = (double*)malloc(sizeof(double) * (size_t)P);
    char* used = (char*)calloc((size_t)S, 1);
    for (int64_t p = 0; p < P; ++p) M[p] = INFINITY;
    for (int t = 0; t < K; ++t) {
        int best = -1;
        double best_area = INFINITY;
        for (int s = 0; s < S; ++s) {
            if (used[s]) continue;
            double a = 0.0;
            for (int64_t p = 0; p < P; ++p) a += fmin(M[p], D[(size_t)s * P + p]);
            if (best < 0 || a < best_area) {
                best = s;
                best_area = a;
            }
        }
        chosen[t] = best;
        area_after[t] = best_area;
        used[best] = 1;
        for (int64_t p = 0; p < P; ++p) M[p] = fmin(M[p], D[(size_t)best * P + p]);
    }
    free(M);
    free(used);
}

/* Nearest snippet of every position (eq. 6, argmin over the K chosen
 * snippets, lowest segment index on ties), each snippet's share of positions
 * (eq. 7) and the eq. 8 order (frac descending, then segment index
 * ascending).  labels[p] is a segment index; order[i] indexes chosen[]. */
void ora_neighbors(const double* D, int64_t P, const int32_t* chosen, int K, int32_t* labels,
                   double* frac, int32_t* order) {
    int64_t* cnt = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    for (int64_t p = 0; p < P; ++p) {
        int bt = -1;
        for (int t = 0; t < K; ++t) {
            double v = D[(size_t)chosen[t] * P + p];
            if (bt < 0) { bt = t; continue; }
            double bv = D[(size_t)chosen[bt] * P + p];
            if (v < bv || (v == bv && chosen[t] < chosen[bt])) bt = t;
        }
        labels[p] = chosen[bt];
        cnt[bt] += 1;
    }
    for (int t = 0; t < K; ++t) frac[t] = (double)cnt[t] / (double)P;
    for (int t = 0; t < K; ++t) order[t] = t;
    /* insertion sort on (frac desc, segment asc) */
    for (int i = 1; i < K; ++i) {
        int32_t x = order[i];
        int j = i - 1;
        while (j >= 0) {
            int32_t y = order[j];
            int before = frac[x] > frac[y] || (frac[x] == frac[y] && chosen[x] < chosen[y]);
            if (!before) break;
            order[j + 1] = y;
            --j;
        }
        order[j + 1] = x;
    }
    free(cnt);
}

/* Length criterion of eq. 18 for one m: the sum over ordered pairs p != q of
 * the chosen snippets of sum_i |D_p(i) - D_q(i)|, divided by the largest
 * profile value over all segments and positions; 0 when that maximum is 0. */
double ora_criterion(const double* D, int S, int64_t P, const int32_t* chosen, int K) {
    double num = 0.0;
    for (int p = 0; p < K; ++p)
        for (int q = 0; q < K; ++q) {
            if (p == q) continue;
            const double* a = D + (size_t)chosen[p] * P;
            const double* b = D + (size_t)chosen[q] * P;
            for (int64_t i = 0; i < P; ++i) num += fabs(a[i] - b[i]);
        }
    double den = 0.0;
    for (size_t i = 0; i < (size_t)S * (size_t)P; ++i) den = fmax(den, D[i]);
    return den > 0.0 ? num / den : 0.0;
}
