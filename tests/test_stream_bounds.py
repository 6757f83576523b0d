"""The lower bounds of the greedy search without the profile set, checked on
the CPU against an oracle profile set (no device).

At greedy step t the area of segment s is A_t(s) = sum_p min(M_t(p), D_s(p))
(eq. 17), M_t the pointwise minimum of the chosen profiles.  On a block of
positions the search bounds it from a sketch of the row taken in one early
pass (block sum A0, largest value X, smallest value N) and, for a row
recomputed at an earlier step ts, from its block area then:
    A >= sum min(M, N)                       (D >= N on the block)
    A >= A0 - sum max(0, X - M)              (D <= X on the block)
    A >= A_ts - (sum M_ts - sum M_t)         (M only shrinks; min is 1-Lipschitz)
Each is restated here from its derivation and must hold block by block, at
every step, for every segment; their sum over blocks bounds the whole area."""
import numpy as np

import oracle
import synth


def _blocks(P, L):
    return [(b, min(P, b + L)) for b in range(0, P, L)]


def test_sketch_bounds_hold_at_every_step():
    rng = np.random.default_rng(21)
    T = synth.random_planted(rng, 5000, 4).T
    m = 64
    D = oracle.profiles(T, m, synth.default_ell(m), synth.default_k(m))
    S, P = D.shape
    blocks = _blocks(P, 200)
    A0 = np.array([[D[s, a:b].sum() for a, b in blocks] for s in range(S)])
    X = np.array([[D[s, a:b].max() for a, b in blocks] for s in range(S)])
    N = np.array([[D[s, a:b].min() for a, b in blocks] for s in range(S)])

    M = np.full(P, np.inf)
    chosen, area_at, curve_sums = [], {}, []
    checked = 0
    for t in range(6):
        area = np.array([np.minimum(M, D[s]).sum() for s in range(S)])
        MB = np.array([M[a:b].sum() for a, b in blocks])
        curve_sums.append(MB)
        for s in range(S):
            if s in chosen:
                continue
            true_blk = np.array([np.minimum(M[a:b], D[s, a:b]).sum() for a, b in blocks])
            if t == 0:
                assert np.allclose(true_blk, A0[s])  # M = +inf: the block sums themselves
                continue
            lbA = np.array([np.minimum(M[a:b], N[s, q]).sum() for q, (a, b) in enumerate(blocks)])
            lbB = np.array([A0[s, q] - np.maximum(0.0, X[s, q] - M[a:b]).sum() for q, (a, b) in enumerate(blocks)])
            tol = 1e-9 * (np.abs(A0[s]) + 1.0)
            assert np.all(lbA <= true_blk + tol) and np.all(lbB <= true_blk + tol)
            if s in area_at:
                ts, blk_ts = area_at[s]
                lbD = blk_ts - (curve_sums[ts] - MB)
                assert np.all(lbD <= true_blk + tol)
            lb = np.maximum(np.maximum(lbA, lbB), 0.0).sum()
            assert lb <= area[s] + 1e-9 * area[s]
            checked += 1
            if rng.random() < 0.3:  # rows "recomputed" at this step keep their block areas
                area_at[s] = (t, true_blk)
        best = int(np.argmin(np.where(np.isin(np.arange(S), chosen), np.inf, area)))
        chosen.append(best)
        M = np.minimum(M, D[best])
    assert checked > 5 * (S - 6)


def test_bounds_are_tight_for_flat_blocks():
    """Where a row is constant on a block (N = X = its value) the first two bounds
    are exact."""
    P, L = 64, 16
    rng = np.random.default_rng(3)
    M = rng.uniform(0.0, 2.0, P)
    d = np.repeat(rng.uniform(0.0, 2.0, P // L), L)
    for a, b in _blocks(P, L):
        v = d[a]
        true = np.minimum(M[a:b], d[a:b]).sum()
        assert np.isclose(np.minimum(M[a:b], v).sum(), true)
        assert np.isclose(d[a:b].sum() - np.maximum(0.0, v - M[a:b]).sum(), true)
