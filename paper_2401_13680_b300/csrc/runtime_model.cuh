// Runtime model of the device work of a length sweep.
//
// Section 4.2 predicts the run time of the snippet search for each length with
// a polynomial regression trained on the times of earlier runs, and uses the
// predictions to spread the lengths over cluster nodes.  On one GPU the same
// kind of model serves the serving engine: it orders admission and waves by
// predicted work (shortest remaining first) and reports predicted times.
//
// A unit of device work (an engine wave, or a whole job) is described by five
// features, and its time in milliseconds is modelled as their dot product with
// five coefficients:
//   f0 = E                  E = eq. 9 cells of the tile launches, in units of 1e9
//   f1 = E * x              (halo columns included), x = m / 256 of each chunk,
//   f2 = E * x^2            summed over the chunks
//   f3 = G                  G = GB of profile set the greedy search reads
//                           (K passes over S x P values per length)
//   f4 = waves              1 per engine wave
// so that c0 + c1 x + c2 x^2 is the cost of 1e9 cells at length m, a quadratic
// in m as in the paper's polynomial regression.  The coefficients are the
// ridge-regularised least-squares fit to every observation so far (normal
// equations), each coefficient pulled toward a prior with a weight of RM_RIDGE
// times its own diagonal entry of the normal matrix (plus 1e-9): the ridge
// does not depend on the features' units, and with few or collinear
// observations (every wave at the same lengths) the directions the data does
// not determine keep the prior's values.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

namespace {

constexpr int RM_NF = 5;
constexpr double RM_RIDGE = 1e-4;

struct RuntimeModel {
    double xtx[RM_NF * RM_NF];
    double xty[RM_NF];
    double coef[RM_NF];
    double prior[RM_NF];
    uint64_t n = 0;         // observations
    double err_sum = 0.0;   // relative errors of predictions made with >= RM_TRAINED observations
    uint64_t err_n = 0;

    void reset(const double* pr) {
        memset(xtx, 0, sizeof xtx);
        memset(xty, 0, sizeof xty);
        memcpy(prior, pr, sizeof prior);
        memcpy(coef, pr, sizeof coef);
        n = 0;
        err_sum = 0.0;
        err_n = 0;
    }

    double predict(const double* f) const {
        double t = 0.0;
        for (int i = 0; i < RM_NF; ++i) t += coef[i] * f[i];
        return t;
    }

    // Solves (X'X + L) c = X'y + L prior, L = diag(RM_RIDGE X'X_ii + 1e-9), by
    // Gaussian elimination with partial pivoting; keeps the old coefficients if
    // the system is singular.
    void refit() {
        double A[RM_NF][RM_NF + 1];
        for (int i = 0; i < RM_NF; ++i) {
            const double lam = RM_RIDGE * xtx[i * RM_NF + i] + 1e-9;
            for (int j = 0; j < RM_NF; ++j) A[i][j] = xtx[i * RM_NF + j] + (i == j ? lam : 0.0);
            A[i][RM_NF] = xty[i] + lam * prior[i];
        }
        for (int c = 0; c < RM_NF; ++c) {
            int p = c;
            for (int r = c + 1; r < RM_NF; ++r)
                if (std::fabs(A[r][c]) > std::fabs(A[p][c])) p = r;
            if (!(std::fabs(A[p][c]) > 0.0)) return;
            if (p != c)
                for (int j = 0; j <= RM_NF; ++j) std::swap(A[p][j], A[c][j]);
            for (int r = c + 1; r < RM_NF; ++r) {
                const double f = A[r][c] / A[c][c];
                for (int j = c; j <= RM_NF; ++j) A[r][j] -= f * A[c][j];
            }
        }
        double x[RM_NF];
        for (int i = RM_NF - 1; i >= 0; --i) {
            double s = A[i][RM_NF];
            for (int j = i + 1; j < RM_NF; ++j) s -= A[i][j] * x[j];
            x[i] = s / A[i][i];
        }
        for (int i = 0; i < RM_NF; ++i)
            if (!std::isfinite(x[i])) return;
        memcpy(coef, x, sizeof coef);
    }

    // One measured unit of work: f its features, ms its time.  `pred` is what
    // the model predicted for it before it ran (< 0: no prediction) and
    // `trained` whether the model had enough data then to count the error.
    void observe(const double* f, double ms, double pred, bool trained) {
        if (!(ms > 0.0) || !std::isfinite(ms)) return;
        for (int i = 0; i < RM_NF; ++i) {
            for (int j = 0; j < RM_NF; ++j) xtx[i * RM_NF + j] += f[i] * f[j];
            xty[i] += f[i] * ms;
        }
        ++n;
        if (trained && pred >= 0.0) {
            err_sum += std::fabs(pred - ms) / ms;
            ++err_n;
        }
        refit();
    }
};

constexpr uint64_t RM_TRAINED = 8;  // observations before predictions count as trained

// Priors: about 11 ms per 1e9 cells in FP32 and 12x that in FP64 (the tile
// kernel's measured sweep rates), 0.25 ms per GB of greedy reads, 0.05 ms per wave.
inline const double* rm_prior(int prec) {
    static const double p32[RM_NF] = {11.0, 0.0, 0.0, 0.25, 0.05};
    static const double p64[RM_NF] = {130.0, 0.0, 0.0, 0.5, 0.05};
    return prec == 1 ? p64 : p32;
}

struct ModelTable {
    std::mutex mu;
    RuntimeModel m[2];
    ModelTable() {
        m[0].reset(rm_prior(0));
        m[1].reset(rm_prior(1));
    }
};

inline ModelTable& rm_table() {
    static ModelTable t;
    return t;
}

// Features of cells eq. 9 cells at length m, added to f.
inline void rm_add_cells(double* f, double cells, int m) {
    const double E = cells * 1e-9, x = (double)m / 256.0;
    f[0] += E;
    f[1] += E * x;
    f[2] += E * x * x;
}

}  // namespace
