"""Tolerance rule for MPdist values (FP32: 1e-4, FP64: 1e-9).

Relative error is ill-posed near d = 0 because d = sqrt(2 ell (1 - rho)) turns a
fixed error in rho into an error in d that grows like ell * d_rho / d.  So the
rule uses a floor d_floor = 0.1 * sqrt(2 ell) (1/20 of the largest possible
distance 2 sqrt(ell)):
    d_ref >= d_floor:  |d - d_ref| <= tol * d_ref
    d_ref <  d_floor:  |d^2 - d_ref^2| <= 2 tol * d_floor^2
The second line is the first one carried into the squared domain at the floor
(a relative error e in d is a relative error 2e in d^2), so the rule is
continuous there; below the floor it allows an error of
2 tol * d_floor^2 / (2 ell) = tol / 50 in rho.
"""
import numpy as np


def d_floor(ell: int) -> float:
    return 0.1 * np.sqrt(2.0 * ell)


def profile_errors(d, d_ref, ell: int):
    """Per-cell error ratio under the rule above (compare with tol)."""
    d = np.asarray(d, dtype=np.float64)
    d_ref = np.asarray(d_ref, dtype=np.float64)
    fl = d_floor(ell)
    above = d_ref >= fl
    ratio = np.empty_like(d_ref)
    ratio[above] = np.abs(d[above] - d_ref[above]) / d_ref[above]
    ratio[~above] = np.abs(d[~above] ** 2 - d_ref[~above] ** 2) / (2.0 * fl ** 2)
    return ratio


def assert_profiles_close(d, d_ref, ell: int, tol: float):
    r = profile_errors(d, d_ref, ell) / tol
    worst = int(np.argmax(r)) if r.size else 0
    assert r.size == 0 or r.max() <= 1.0, (
        f"worst cell {np.unravel_index(worst, np.shape(d_ref))}: got {np.ravel(d)[worst]!r}, "
        f"oracle {np.ravel(d_ref)[worst]!r}, error/tol = {r.ravel()[worst]:.3g}, "
        f"cells over: {int((r > 1).sum())} of {r.size}")
    return float(r.max()) if r.size else 0.0


# The FP32 path also meets the rule's below-floor bound in rho everywhere:
# |rho - rho_ref| <= tol / 50 (2e-6 at tol = 1e-4), i.e. |d^2 - d_ref^2| <=
# 2 ell tol / 50.  Above the floor that is stricter than the relative bound on
# d; the greedy search's FP64 re-evaluation of near-tied steps bounds its FP32
# areas with it.
RHO_TOL = 2e-6


def rho_errors(d, d_ref, ell: int):
    d = np.asarray(d, dtype=np.float64)
    d_ref = np.asarray(d_ref, dtype=np.float64)
    return np.abs(d ** 2 - d_ref ** 2) / (2.0 * ell)


def assert_rho_close(d, d_ref, ell: int, tol: float = RHO_TOL):
    r = rho_errors(d, d_ref, ell)
    worst = int(np.argmax(r)) if r.size else 0
    assert r.size == 0 or r.max() <= tol, (
        f"worst cell {np.unravel_index(worst, np.shape(d_ref))}: |d rho| = {r.ravel()[worst]:.3g} > {tol:g}, "
        f"cells over: {int((r > tol).sum())} of {r.size}")
    return float(r.max()) if r.size else 0.0
