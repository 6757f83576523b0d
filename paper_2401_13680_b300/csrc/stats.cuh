// ell-window statistics (FP64) and the terms of the centred covariance recurrence.
//
// For every ell-window j of T (j = 0 .. C-1, C = n - ell + 1):
//   mu[j]  mean of T[j .. j+ell)
//   a[j]   1 / sqrt(sum_t (T[j+t] - mu[j])^2) = 1 / (sqrt(ell) * sigma_j), population sigma;
//          0 for a flat window (centred sum of squares <= 1e-24 * ell * max(1, mu^2))
//   df[j]  (T[j+ell-1] - T[j-1]) / 2                                   (0 for j = 0)
//   dg[j]  (T[j+ell-1] - mu[j]) + (T[j-1] - mu[j-1])                   (0 for j = 0)
// so that the centred covariance cov(i, j) = sum_t (T[i+t]-mu_i)(T[j+t]-mu_j) obeys
//   cov(i, j) = cov(i-1, j-1) + df[i] * dg[j] + df[j] * dg[i]
// and the Pearson correlation is rho(i, j) = cov(i, j) * a[i] * a[j]; the
// z-normalised distance is sqrt(2 ell (1 - rho)) (Section 4.1: the dot-product
// technique of the matrix-profile work the paper cites as [7]).
//
// The tile kernel works in the precision `real` only (FP64 arithmetic is slow
// on this GPU), so the FP64 series and means are also kept as unevaluated
// pairs hi + lo of `real` values (hi = the rounded value, lo = the rounded
// remainder): Th, Tl for T (n values) and muh, mul for mu (C values).  In the
// FP64 path hi is the value itself and lo is 0.
#pragma once
#include <cstdint>

namespace pastila {

constexpr int STATS_RUN = 32;  // windows per thread; sums restart at every run

// Run-local prefix sums: each thread sums its first window directly about a local
// reference value, then slides the sums across STATS_RUN windows.  A window whose
// slid centred sum of squares looks small is recomputed two-pass so that the
// flatness decision is taken on an exact-as-possible value.
__global__ void stats_mu_a_kernel(const double* __restrict__ T, int64_t C, int ell,
                                  double* __restrict__ mu, double* __restrict__ inv_norm,
                                  int32_t* __restrict__ flat) {
    const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * STATS_RUN;
    if (j0 >= C) return;
    const double ref = T[j0];
    double s1 = 0.0, s2 = 0.0;
    for (int t = 0; t < ell; ++t) {
        const double d = T[j0 + t] - ref;
        s1 += d;
        s2 += d * d;
    }
    const int64_t jend = j0 + STATS_RUN < C ? j0 + STATS_RUN : C;
    for (int64_t j = j0; j < jend; ++j) {
        if (j > j0) {
            const double dout = T[j - 1] - ref, din = T[j + ell - 1] - ref;
            s1 += din - dout;
            s2 += din * din - dout * dout;
        }
        const double mloc = s1 / ell;
        const double m = ref + mloc;
        double ss = s2 - s1 * mloc;
        const double scale = m * m > 1.0 ? m * m : 1.0;
        if (ss <= 1e-10 * ell * scale) {  // small: recompute two-pass
            double mm = 0.0;
            for (int t = 0; t < ell; ++t) mm += T[j + t];
            mm /= ell;
            double acc = 0.0;
            for (int t = 0; t < ell; ++t) acc += (T[j + t] - mm) * (T[j + t] - mm);
            ss = acc;
        }
        const int f = ss <= 1e-24 * ell * scale;
        mu[j] = m;
        inv_norm[j] = f ? 0.0 : 1.0 / sqrt(ss);
        flat[j] = f;
    }
}

template <typename real>
__device__ __forceinline__ void split2(double x, real* hi, real* lo) {
    const real h = (real)x;
    *hi = h;
    *lo = (real)(x - (double)h);
}

// Grid over the n values of T: j < n writes the pair of T[j], j < C the
// statistics of window j.
template <typename real>
__global__ void stats_terms_kernel(const double* __restrict__ T, int64_t n, int64_t C, int ell,
                                   const double* __restrict__ mu,
                                   const double* __restrict__ inv_norm, real* __restrict__ a,
                                   real* __restrict__ df, real* __restrict__ dg, real* __restrict__ muh,
                                   real* __restrict__ mul, real* __restrict__ Th, real* __restrict__ Tl) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) split2(T[j], Th + j, Tl + j);
    if (j >= C) return;
    split2(mu[j], muh + j, mul + j);
    a[j] = (real)inv_norm[j];
    if (j == 0) {
        df[j] = (real)0;
        dg[j] = (real)0;
    } else {
        const double tin = T[j + ell - 1], tout = T[j - 1];
        df[j] = (real)((tin - tout) * 0.5);
        dg[j] = (real)((tin - mu[j]) + (tout - mu[j - 1]));
    }
}

// Conditioning of the FP32 covariance recurrence (FP32 tiles).  Along a
// diagonal the recurrence accumulates rounding errors at the scale of the
// windows it passed through, while rho divides by the norms of the current
// ones: a cell (i, j) whose windows are much smaller than those of the last R
// steps of its diagonal can lose the FP32 accuracy the tolerance rule asks
// (|d rho| <= 2e-6).  kappa[j] = a[j] / min{a[u] > 0 : max(0, j-R+1) <= u <= j}
// (the largest norm among the R windows up to j over the norm of window j;
// 0 for a flat window, whose rho the flat rule sets) bounds that ratio for
// the row and the column side alike; the tile recomputes a cell exactly when
// kappa[i] * kappa[j] exceeds KAPPA_FLAG (the recurrence's error in rho grows
// about in proportion to that product).  One thread per
// window; R loads each (a few hundred), once per length.
template <typename real>
__global__ void kappa_kernel(const real* __restrict__ a, int64_t C, int R, float* __restrict__ kappa) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= C) return;
    const real aj = a[j];
    if (!(aj > (real)0)) {
        kappa[j] = 0.0f;
        return;
    }
    real mn = aj;
    const int64_t u0 = j - R + 1 > 0 ? j - R + 1 : 0;
    for (int64_t u = u0; u < j; ++u) {
        const real au = a[u];
        if (au > (real)0 && au < mn) mn = au;
    }
    kappa[j] = (float)(aj / mn);
}

}  // namespace pastila
