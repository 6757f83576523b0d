"""Pins of the FP64 oracle against things other than itself: library routines
(numpy / scipy), brute force on tiny inputs, closed forms, special cases and
invariants the definitions imply.  CPU only."""
import math

import numpy as np
import pytest
from scipy.spatial.distance import cdist
from scipy.stats import zscore

import oracle
import synth


def _z_windows(x, ell):
    w = np.lib.stride_tricks.sliding_window_view(np.asarray(x, float), ell)
    return zscore(w, axis=1, ddof=0)


def _mpdist_brute(A, B, ell, k):
    """MPdist from its definition with scipy: all ell-subsequence distances of
    z-normalised windows, row minima ++ column minima, k-th smallest (1-based)
    or the maximum when there are at most k values."""
    E = cdist(_z_windows(A, ell), _z_windows(B, ell))
    v = np.sort(np.concatenate([E.min(axis=1), E.min(axis=0)]))
    return v[k - 1] if v.size > k else v[-1]


# --------------------------------------------------------------------------- stats / distance

def test_window_stats_match_numpy():
    T = synth.white_noise(3, 500) * 3 + 7
    for ell in (2, 5, 64):
        mu, sig, flat = oracle.window_stats(T, ell)
        w = np.lib.stride_tricks.sliding_window_view(T, ell)
        np.testing.assert_allclose(mu, w.mean(axis=1), rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(sig, w.std(axis=1, ddof=0), rtol=1e-12)
        assert not flat.any()


def test_window_stats_flat_flag():
    T = np.concatenate([np.full(20, 3.25), synth.white_noise(1, 20)])
    mu, sig, flat = oracle.window_stats(T, 8)
    assert flat[:13].all() and not flat[13:].any()


def test_zdist_matches_scipy_and_closed_form():
    rng = np.random.default_rng(4)
    for ell in (3, 16, 100):
        x, y = rng.normal(size=ell) * 5 + 1, rng.normal(size=ell) - 2
        ref = np.linalg.norm(zscore(x) - zscore(y))
        d = oracle.zdist(x, y)
        assert d == pytest.approx(ref, rel=1e-12)
        rho = np.corrcoef(x, y)[0, 1]
        assert d * d == pytest.approx(2 * ell * (1 - rho), rel=1e-10)


def test_zdist_flat_rule():
    ell = 10
    flat, other = np.full(ell, 2.0), np.arange(ell, dtype=float)
    assert oracle.zdist(flat, flat * 3) == 0.0
    assert oracle.zdist(flat, other) == pytest.approx(math.sqrt(2 * ell))


# --------------------------------------------------------------------------- MPdist

@pytest.mark.parametrize("m,ell,k", [(16, 8, 2), (16, 8, 1), (20, 5, 7), (12, 11, 3), (9, 9, 4),
                                     (24, 12, 30), (10, 3, 16)])
def test_mpdist_pair_matches_brute_force(m, ell, k):
    rng = np.random.default_rng(m * 100 + ell * 10 + k)
    for _ in range(5):
        A, B = rng.normal(size=m).cumsum(), rng.normal(size=m).cumsum()
        assert oracle.mpdist(A, B, ell, k) == pytest.approx(_mpdist_brute(A, B, ell, k), rel=1e-11)


def test_mpdist_ell_equals_m_is_znorm_distance():
    # R = 1: P_ABBA holds the same distance twice and k >= 2 selects the maximum,
    # so MPdist is the z-normalised Euclidean distance of the whole windows.
    rng = np.random.default_rng(7)
    for m in (8, 33, 128):
        A, B = rng.normal(size=m), rng.normal(size=m) * 2 + 1
        ref = np.linalg.norm(zscore(A) - zscore(B))
        assert oracle.mpdist(A, B, m, (m + 9) // 10) == pytest.approx(ref, rel=1e-12)


def test_mpdist_k1_is_min_distance():
    rng = np.random.default_rng(8)
    A, B = rng.normal(size=30), rng.normal(size=30)
    ref = cdist(_z_windows(A, 10), _z_windows(B, 10)).min()
    assert oracle.mpdist(A, B, 10, 1) == pytest.approx(ref, rel=1e-12)


def test_mpdist_symmetry_and_identity():
    rng = np.random.default_rng(9)
    A, B = rng.normal(size=40), rng.normal(size=40)
    assert oracle.mpdist(A, B, 20, 4) == pytest.approx(oracle.mpdist(B, A, 20, 4), rel=1e-13)
    assert oracle.mpdist(A, A, 20, 4) == pytest.approx(0.0, abs=1e-6)


# --------------------------------------------------------------------------- profiles (eqs. 9-15)

@pytest.mark.parametrize("n,m,ell,k", [(96, 16, 8, 2), (100, 16, 8, 2), (130, 20, 7, 5),
                                        (64, 8, 8, 2), (90, 12, 4, 25)])
def test_psf_profiles_equal_pair_definition(n, m, ell, k):
    """The PSF steps (column minima, row windows of m-ell+1 columns, concatenation
    with allP_BA(p .. p+m-ell), k-th) give the pair-definition MPdist at every
    (segment, position): pins the index readings of eqs. 11-13."""
    T = synth.white_noise(n, n).cumsum()
    D = oracle.profiles(T, m, ell, k)
    S, P = n // m, n - m + 1
    assert D.shape == (S, P)
    segs, pos = np.meshgrid(np.arange(S), np.arange(P), indexing="ij")
    ref = oracle.profile_cells(T, m, ell, k, segs.ravel(), pos.ravel()).reshape(S, P)
    np.testing.assert_allclose(D, ref, rtol=1e-12, atol=1e-12)
    # and against scipy brute force on a few cells
    for s, p in [(0, 0), (S - 1, P - 1), (1, 3)]:
        assert D[s, p] == pytest.approx(_mpdist_brute(T[s * m:s * m + m], T[p:p + m], ell, k),
                                        rel=1e-11, abs=1e-12)


def test_profile_invariants():
    n, m, ell, k = 240, 24, 12, 5
    T = synth.white_noise(11, n) + np.sin(np.arange(n) / 3.0)
    D = oracle.profiles(T, m, ell, k)
    S, P = D.shape
    for s in range(S):
        assert abs(D[s, s * m]) < 1e-6                       # zero at own offset
    assert (D >= 0).all() and (D <= 2 * math.sqrt(ell) + 1e-12).all()
    # affine maps a T + b, a != 0: both windows of every pair change together,
    # so z-normalised distances (and D) are unchanged, negative a included
    for a, b in ((2.5, -7.0), (-3.5, 12.0)):
        np.testing.assert_allclose(oracle.profiles(a * T + b, m, ell, k), D, rtol=1e-9, atol=1e-9)
    Dr = oracle.profiles(T[::-1].copy(), m, ell, k)         # time reversal (m divides n)
    np.testing.assert_allclose(Dr[::-1, ::-1], D, rtol=1e-9, atol=1e-9)


def test_periodic_series_zero_at_period_lags():
    # noise-free sine whose period divides m: every segment equals the window at
    # any lag that is a multiple of the period, so D is 0 there; with fewer
    # ell-subsequences per window (R = 9) than phases in a period (64), the
    # half-period lag matches no phase and stays far from 0
    period, m, ell = 64, 128, 120
    T = np.sin(2 * np.pi * np.arange(1280) / period)
    D = oracle.profiles(T, m, ell, 2)
    for s in range(D.shape[0]):
        assert np.max(np.abs(D[s, ::period])) < 1e-5
        assert D[s, period // 2] > 1.0


def test_planted_regimes_recovered():
    s = synth.four_regimes()
    chosen, area, labels, frac, order, D = oracle.snippets(s.T, 128, 64, 13, 4)
    regimes = {s.regime_of(int(c) * 128) for c in chosen}
    assert len(regimes) == 4
    assert np.all(np.diff(area) <= 0)


# --------------------------------------------------------------------------- greedy (eqs. 16-17)

def _greedy_brute(D, K):
    S, P = D.shape
    M = np.full(P, np.inf)
    chosen, areas = [], []
    for _ in range(K):
        best, best_a = None, None
        for s in range(S):
            if s in chosen:
                continue
            a = sum(min(M[p], D[s, p]) for p in range(P))
            if best is None or a < best_a:
                best, best_a = s, a
        chosen.append(best)
        areas.append(best_a)
        M = np.minimum(M, D[best])
    return chosen, areas


def test_greedy_hand_case():
    D = np.array([[0.0, 4.0, 4.0, 4.0],
                  [4.0, 0.0, 1.0, 4.0],
                  [3.0, 3.0, 0.0, 0.0],
                  [1.0, 1.0, 1.0, 1.0]])
    chosen, area = oracle.greedy(D, 3)
    # step 1 row sums: 12, 9, 6, 4 -> segment 3 (area 4)
    # step 2 with M = 1,1,1,1: s0 -> 0+1+1+1 = 3, s1 -> 1+0+1+1 = 3, s2 -> 1+1+0+0 = 2
    # step 3 with M = 1,1,0,0: s0 -> 0+1 = 1, s1 -> 1+0 = 1 -> tie, lowest index 0
    assert list(chosen) == [3, 2, 0]
    np.testing.assert_allclose(area, [4.0, 2.0, 1.0])


def test_greedy_matches_python_loops():
    rng = np.random.default_rng(12)
    for _ in range(5):
        D = rng.integers(0, 5, size=(7, 23)).astype(float)   # many ties
        c, a = oracle.greedy(D, 5)
        cb, ab = _greedy_brute(D, 5)
        assert list(c) == cb
        np.testing.assert_allclose(a, ab)
        assert np.argmin(D.sum(axis=1)) == c[0]


# --------------------------------------------------------------------------- neighbours (eqs. 6-8)

def test_neighbors_hand_case():
    D = np.array([[0.0, 2.0, 5.0, 1.0, 3.0],
                  [9.0, 9.0, 9.0, 9.0, 9.0],
                  [1.0, 2.0, 0.0, 1.0, 3.0]])
    labels, frac, order = oracle.neighbors(D, [2, 0])
    # p0 -> seg0 (0<1); p1 tie 2=2 -> lowest segment 0; p2 -> seg2; p3 tie -> 0; p4 tie -> 0
    assert list(labels) == [0, 0, 2, 0, 0]
    np.testing.assert_allclose(frac, [0.2, 0.8])            # per chosen: seg2, seg0
    assert list(order) == [1, 0]                             # seg0 first (larger frac)
    assert frac.sum() == pytest.approx(1.0)


def test_neighbors_frac_tie_order():
    D = np.array([[0.0, 1.0], [1.0, 0.0]])
    labels, frac, order = oracle.neighbors(D, [1, 0])
    np.testing.assert_allclose(frac, [0.5, 0.5])
    assert list(order) == [1, 0]                             # equal frac: segment 0 first


# --------------------------------------------------------------------------- criterion (eq. 18)

def test_criterion_closed_form():
    D = np.array([[1.0, 2.0, 3.0],
                  [3.0, 2.0, 1.0],
                  [0.0, 0.0, 4.0]])
    # ordered pairs (0,1),(1,0): 2 * (2 + 0 + 2) = 8; max over all of D = 4
    assert oracle.criterion(D, [0, 1]) == pytest.approx(2.0)
    # three snippets: |d01| = 4, |d02| = 1+2+1 = 4, |d12| = 3+2+3 = 8 -> 2*16/4
    assert oracle.criterion(D, [0, 1, 2]) == pytest.approx(8.0)
    assert oracle.criterion(D, [1]) == 0.0
    assert oracle.criterion(D * 7.0, [0, 1]) == pytest.approx(2.0)
    assert oracle.criterion(np.zeros((2, 3)), [0, 1]) == 0.0


def test_select_length_argmax_smallest_on_tie():
    s = synth.four_regimes(per_regime=256)
    ms = [32, 48, 64]
    m_best, crit, chosen = oracle.select_length(s.T, ms, 2, lambda m: m // 2,
                                                lambda m: (m + 9) // 10)
    assert crit.shape == (3,)
    assert m_best == ms[int(np.argmax(crit))]
    for m in ms:
        D = oracle.profiles(s.T, m, m // 2, (m + 9) // 10)
        c, _ = oracle.greedy(D, 2)
        assert crit[ms.index(m)] == pytest.approx(oracle.criterion(D, c))


# --------------------------------------------------------------------------- stored values

def test_golden_fixtures_reproduce():
    import json, os
    here = os.path.join(os.path.dirname(__file__), "golden")
    g = json.load(open(os.path.join(here, "four_regimes_m128.json")))
    s = synth.four_regimes()
    D = oracle.profiles(s.T, g["m"], g["ell"], g["k"])
    assert D.max() == pytest.approx(g["D_max"], rel=1e-12)
    for a, b, v in g["cells"]:
        assert D[a, b] == pytest.approx(v, rel=1e-12, abs=1e-12)
    for K in (2, 4):
        c, area = oracle.greedy(D, K)
        assert list(c) == g[f"K{K}"]["chosen"]
    t = json.load(open(os.path.join(here, "tiny_walk_m24.json")))
    T = synth.white_noise(77, 120).cumsum()
    np.testing.assert_allclose(oracle.profiles(T, t["m"], t["ell"], t["k"]), np.array(t["D"]),
                               rtol=1e-12, atol=1e-12)


def test_profiles_range_matches_full():
    T = synth.white_noise(21, 400).cumsum()
    D = oracle.profiles(T, 32, 16, 4)
    segs = [0, 5, 11]
    np.testing.assert_array_equal(oracle.profiles_range(T, 32, 16, 4, segs, 17, 201), D[segs, 17:201])

