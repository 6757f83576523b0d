"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  FP32 profiles within 1e-4, FP64 within 1e-9, under the
floor rule of tests/tolerance.py; snippet indices bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from tolerance import assert_profiles_close, assert_rho_close

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-9}


def _series(T, prec):
    from paper_2401_13680_b300 import pastila
    return pastila.Series(T, precision=prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_four_regime_profiles(lib, prec):
    s = synth.four_regimes()
    m, ell, k = 128, 64, 13
    ref = oracle.profiles(s.T, m, ell, k)
    with _series(s.T, prec) as h:
        D, dmax = h.profiles(m)
    assert D.shape == ref.shape
    assert_profiles_close(D, ref, ell, TOL[prec])
    if prec == 0:
        assert_rho_close(D, ref, ell)
    assert dmax == pytest.approx(ref.max(), rel=TOL[prec])


# (n, m, ell, k): several tiles with a ragged last tile and a tail segment
# (n % m != 0); R < V (ell close to m); R = 1 (ell = m); k >= 2R (max branch);
# k = 1 (min branch); odd sizes; R > 288 and R > 384 (the selection keeps 12
# values of a column per lane in registers and reads the rest from shared memory);
# odd m, so that segment starts s m fall at every offset from a 16-byte boundary
# (the tile stages segment data from the boundary below the start)
CASES = [
    (2777, 77, 39, 8),
    (1999, 33, 17, 4),
    (4000, 640, 320, 64),
    (4500, 600, 150, 60),
    (3000, 400, 200, 40),
    (3000, 64, 32, 7),
    (2501, 50, 25, 5),
    (1800, 40, 37, 3),
    (1500, 30, 30, 3),
    (1200, 24, 20, 12),
    (1700, 48, 16, 1),
    (5003, 100, 50, 10),
    (900, 8, 4, 2),
]


@pytest.mark.parametrize("n,m,ell,k", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_profiles_shapes_and_edges(lib, n, m, ell, k, prec):
    """Tile, tail and selection logic on planted regimes (both precisions; the
    FP32 tiles recompute the cells whose windows are far smaller than those on
    their diagonal's history) and, FP32, on a random walk plus noise.  FP32 also
    meets 2e-6 in rho at every cell."""
    rng = np.random.default_rng(n + m)
    inputs = [synth.random_planted(rng, n, 3).T]
    if prec == 0:
        inputs.append(np.cumsum(rng.normal(0, 0.2, n)) + rng.normal(0, 1.0, n))
    for T in inputs:
        ref = oracle.profiles(T, m, ell, k)
        with _series(T, prec) as h:
            D, dmax = h.profiles(m, ell=ell, k=k)
        assert_profiles_close(D, ref, ell, TOL[prec])
        if prec == 0:
            assert_rho_close(D, ref, ell)


@pytest.mark.parametrize("prec", [0, 1])
def test_random_walk_with_drift(lib, prec):
    # wandering mean (the drift workload's character) stresses the shifted seeds
    rng = np.random.default_rng(5)
    T = np.cumsum(rng.normal(0, 0.3, 6000)) + 50.0
    m, ell, k = 96, 48, 10
    ref = oracle.profiles(T, m, ell, k)
    with _series(T, prec) as h:
        D, _ = h.profiles(m)
    assert_profiles_close(D, ref, ell, TOL[prec])


def _flat_series():
    rng = np.random.default_rng(9)
    T = rng.normal(size=1200)
    T[300:420] = 2.5      # flat stretches longer than ell: flat windows on both sides
    T[800:860] = -1.0
    return T


def test_flat_windows_fp64(lib):
    T = _flat_series()
    m, ell, k = 40, 20, 4
    ref = oracle.profiles(T, m, ell, k)
    with _series(T, 1) as h:
        D, _ = h.profiles(m)
    assert_profiles_close(D, ref, ell, TOL[1])


def test_flat_windows_fp32(lib):
    """The flat rule holds exactly in FP32 (two flat windows at distance 0, a
    flat and a non-flat one at sqrt(2 ell)), and every cell, those whose windows
    straddle a flat edge included, meets the FP32 tolerance."""
    T = _flat_series()
    m, ell, k = 40, 20, 4
    ref = oracle.profiles(T, m, ell, k)
    with _series(T, 0) as h:
        D, _ = h.profiles(m)
    exact = (ref == 0.0) | (ref == np.sqrt(2.0 * ell))
    assert np.all(D[exact] == ref[exact].astype(np.float32))
    assert_profiles_close(D, ref, ell, TOL[0])
    assert_rho_close(D, ref, ell)


def test_fp32_ill_conditioned_windows(lib):
    """Where a window's spread is far below that of the windows before it on
    its diagonal (4-sample windows at the flat foot of a bump train; windows
    with one informative sample at a flat edge), the FP32 recurrence would keep
    an absolute error set by the larger spread (1.1e-5 and 2.1e-5 in rho on
    these inputs, 5x and 10x the allowance); the tiles recompute those cells by
    exact dot products, and every cell meets the rule."""
    cases = [(synth.random_planted(np.random.default_rng(908), 900, 3).T, 8, 4, 2),
             (_flat_series(), 40, 20, 4)]
    for T, m, ell, k in cases:
        ref = oracle.profiles(T, m, ell, k)
        with _series(T, 0) as h:
            D, _ = h.profiles(m)
        assert_profiles_close(D, ref, ell, TOL[0])
        assert_rho_close(D, ref, ell)


def test_fp32_own_offset_is_zero(lib):
    s = synth.four_regimes()
    with _series(s.T, 0) as h:
        D, _ = h.profiles(128)
    own = D[np.arange(D.shape[0]), np.arange(D.shape[0]) * 128]
    assert np.all(own == 0.0)


@pytest.mark.parametrize("prec", [0, 1])
def test_deterministic(lib, prec):
    s = synth.four_regimes()
    with _series(s.T, prec) as h:
        D1, m1 = h.profiles(128)
        D2, m2 = h.profiles(128)
    assert np.array_equal(D1, D2) and m1 == m2


@pytest.mark.parametrize("K", [2, 4])
def test_snippets_fp64_bit_exact(lib, K):
    s = synth.four_regimes()
    m, ell, k = 128, 64, 13
    chosen, area, labels, frac, order, D = oracle.snippets(s.T, m, ell, k, K)
    with _series(s.T, 1) as h:
        recs, lab, prof = h.snippets(m, K, want_labels=True, want_profiles=True)
    assert [r[0] for r in recs] == [int(chosen[o]) for o in order]
    assert [r[1] for r in recs] == [int(o) for o in order]
    np.testing.assert_allclose([r[2] for r in recs], [frac[o] for o in order], rtol=0, atol=0)
    np.testing.assert_allclose([r[3] for r in recs], [area[o] for o in order], rtol=1e-9)
    assert np.array_equal(lab, labels)
    np.testing.assert_allclose(prof, D[chosen], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_snippets_every_segment_chosen(lib, prec):
    # K = S: every segment becomes a snippet, in the FP64 oracle's greedy order
    # (FP32: near-tied steps, frequent here, are decided on FP64 areas); FP64
    # also the oracle's areas, shares and labels.  The areas never grow.
    from paper_2401_13680_b300 import pastila
    s = synth.four_regimes(per_regime=320)  # n = 1280
    m, ell, k = 128, 64, 13
    S = s.T.shape[0] // m
    with pastila.Series(s.T, precision=prec) as h:
        recs, lab, prof = h.snippets(m, S, want_labels=True, want_profiles=True)
    chosen, area, labels, frac, order, Dr = oracle.snippets(s.T, m, ell, k, S)
    by_step = sorted(recs, key=lambda r: r[1])
    assert sorted(r[0] for r in recs) == list(range(S))
    assert [r[0] for r in by_step] == [int(c) for c in chosen]
    if prec == 1:
        assert [r[0] for r in recs] == [int(chosen[o]) for o in order]
        np.testing.assert_allclose([r[2] for r in recs], [frac[o] for o in order], rtol=0, atol=1e-12)
        np.testing.assert_allclose([r[3] for r in recs], [area[o] for o in order], rtol=1e-9)
        assert np.array_equal(lab, labels)
    else:
        np.testing.assert_allclose([r[3] for r in by_step], area, rtol=3e-4, atol=1e-9)
        _assert_labels_agree(lab, chosen, Dr, ell)
    assert all(b[3] <= a_[3] for a_, b in zip(by_step, by_step[1:]))


def _value_bound(d, ell, tol=1e-4):
    """Largest |d32 - d64| the tolerance rule allows for an FP32 value d."""
    fl = 0.1 * np.sqrt(2.0 * ell)
    c = 2.2 * tol * fl * fl
    return np.where(d >= fl, tol * d, c / (np.sqrt(d * d + c) + d) + tol * fl)


def _assert_labels_agree(lab, chosen, Dref, ell):
    """Labels equal the oracle's except where the two nearest chosen FP64
    profiles are within the FP32 tolerance of each other (either label is then
    a correct reading of FP32 values)."""
    ref_lab, _, _ = oracle.neighbors(Dref, chosen)
    diff = lab != ref_lab
    if diff.any():
        prof = np.sort(Dref[chosen][:, diff], axis=0)
        assert np.all(prof[1] - prof[0] <= _value_bound(prof[0], ell) + _value_bound(prof[1], ell)), \
            int(diff.sum())
    assert diff.mean() < 1e-3


@pytest.mark.parametrize("K", [2, 4])
def test_snippets_fp32(lib, K):
    """FP32 snippet indices equal the FP64 oracle's, step by step: a greedy step
    whose FP32 areas leave more than one segment within their error bounds of
    the minimum is decided on FP64 areas of FP64 rows.  Labels agree except at
    near-ties of the two nearest snippets."""
    s = synth.four_regimes()
    m, ell, k = 128, 64, 13
    chosen, area, labels, frac, order, Dr = oracle.snippets(s.T, m, ell, k, K)
    with _series(s.T, 0) as h:
        recs, lab, prof = h.snippets(m, K, want_labels=True, want_profiles=True)
    by_step = sorted(recs, key=lambda r: r[1])
    assert [r[0] for r in by_step] == [int(c) for c in chosen]
    np.testing.assert_allclose([r[3] for r in by_step], area, rtol=3e-4)
    _assert_labels_agree(lab, chosen, Dr, ell)
    assert sorted(r[0] for r in recs) == sorted(int(c) for c in chosen)


@pytest.mark.parametrize("prec", [0, 1])
def test_select_length_small_sweep(lib, prec):
    s = synth.four_regimes(per_regime=512)
    ms = [32, 48, 64, 80]
    K = 3
    m_best, crit, chosen = oracle.select_length(s.T, ms, K, lambda m: m // 2, lambda m: (m + 9) // 10)
    with _series(s.T, prec) as h:
        gb, gcrit, recs = h.select_length(ms, K)
        per_m = {m: h.snippets(m, K)[0] for m in ms}
    # criterion: relative error of a sum of |differences| of profiles, each within tol
    np.testing.assert_allclose(gcrit, crit, rtol=1e-3 if prec == 0 else 1e-8)
    assert gb == m_best
    assert [r[0] for r in sorted(recs, key=lambda r: r[1])] == [int(c) for c in chosen[m_best]]
    for m in ms:  # the snippets of every length, in greedy order
        assert [r[0] for r in sorted(per_m[m], key=lambda r: r[1])] == [int(c) for c in chosen[m]], m


def test_select_length_reduced_six_regime_sweep(lib):
    """The benchmark's six-regime sweep reduced to n = 20,000 (all 15 lengths
    m = 64 .. 512, ell = m/2, K = 4), FP32: m_best, its snippets and every
    length's snippets equal the FP64 oracle's; the criterion within 1e-3."""
    T = synth.six_regime_sweep(n=20_000, min_len=1500).T
    ms, K = synth.sweep_lengths(), 4
    m_best, crit, chosen = oracle.select_length(T, ms, K, lambda m: m // 2, lambda m: (m + 9) // 10)
    with _series(T, 0) as h:
        gb, gcrit, recs = h.select_length(ms, K)
        per_m = {m: h.snippets(m, K)[0] for m in ms}
    np.testing.assert_allclose(gcrit, crit, rtol=1e-3)
    assert gb == m_best
    assert [r[0] for r in sorted(recs, key=lambda r: r[1])] == [int(c) for c in chosen[m_best]]
    for m in ms:
        assert [r[0] for r in sorted(per_m[m], key=lambda r: r[1])] == [int(c) for c in chosen[m]], m


def test_sweep_full_size_sampled_cells(lib):
    """The n = 100,000 six-regime sweep at full size, in the FP32 configuration the
    benchmark times: 200 sampled (segment, position) cells per m checked against
    the pair definition, for three lengths of the sweep."""
    s = synth.six_regime_sweep()
    rng = np.random.default_rng(123)
    with _series(s.T, 0) as h:
        for m in (64, 256, 512):
            ell, k = m // 2, (m + 9) // 10
            D, dmax = h.profiles(m)
            S, P = D.shape
            segs = rng.integers(0, S, 200)
            pos = rng.integers(0, P, 200)
            pos[:8] = [0, P - 1, P - 2, 1, segs[0] * m, segs[1] * m, P // 2, P // 3]
            ref = oracle.profile_cells(s.T, m, ell, k, segs, pos)
            assert_profiles_close(D[segs, pos], ref, ell, TOL[0])
            assert np.all(D >= 0) and np.all(D <= 2 * np.sqrt(ell) * (1 + 1e-6))
            assert dmax == pytest.approx(float(D.max()), rel=1e-7)


def test_batched_sweep_launch_full_size(lib):
    """The launch the benchmark times, at full size: the six-regime sweep
    (n = 100,000, all 15 lengths, tile layouts tuned as the benchmark tunes them)
    through pastila_profiles_batch_device, which runs select_length's batched
    tile launch into caller buffers.  Every length's profile set equals the
    single-length launch's bit for bit, and on every length seeded cells plus
    both sides of tile boundaries, the first and last position and the first and
    last segment meet the FP32 rule against the oracle (and |d rho| <= 2e-6)."""
    import torch
    from paper_2401_13680_b300 import pastila
    s = synth.six_regime_sweep()
    T = s.T
    n = T.shape[0]
    ms = synth.sweep_lengths()
    rng = np.random.default_rng(2024)
    dev = torch.device("cuda", 0)
    pastila.tune_clear()
    try:
        with pastila.Series(T, precision=0) as h:
            h.tune(ms, max_candidates=4)
            bufs = [torch.empty((n // m) * (n - m + 1), dtype=torch.float32, device=dev) for m in ms]
            dmax = torch.zeros(len(ms), dtype=torch.float64, device=dev)
            h.profiles_batch_device(ms, [b.data_ptr() for b in bufs], dmax.data_ptr())
            torch.cuda.synchronize()
            h.stage_status()
            one = torch.empty_like(bufs[0])
            one_max = torch.zeros(1, dtype=torch.float64, device=dev)
            for i, m in enumerate(ms):
                ell, k = m // 2, (m + 9) // 10
                S, P = n // m, n - m + 1
                h.profiles_device(m, one.data_ptr(), one_max.data_ptr())
                torch.cuda.synchronize()
                assert torch.equal(one[:S * P], bufs[i]), m
                assert one_max.item() == dmax[i].item()
                W = h.tile_layout(m)["W"]
                segs = list(rng.integers(0, S, 24)) + [0, S - 1, 0, S - 1]
                pos = list(rng.integers(0, P, 24)) + [0, P - 1, P - 1, 0]
                for b in range(W, min(P, 9 * W), W):
                    segs += [int(rng.integers(0, S))] * 2
                    pos += [b - 1, b]
                segs = np.array(segs, dtype=np.int32)
                pos = np.array(pos, dtype=np.int64)
                idx = torch.from_numpy(segs.astype(np.int64) * P + pos).to(dev)
                got = bufs[i][idx].double().cpu().numpy()
                ref = oracle.profile_cells(T, m, ell, k, segs, pos)
                assert_profiles_close(got, ref, ell, TOL[0])
                assert_rho_close(got, ref, ell)
                assert dmax[i].item() == pytest.approx(float(bufs[i][:S * P].max()), rel=1e-7)
    finally:
        pastila.tune_clear()


def test_select_length_batched_graph_replay(lib):
    """FP32 select_length runs every length in batched launches, is captured in a
    CUDA graph on its second call and replayed after: three calls agree bit for
    bit; each criterion equals eq. 18 evaluated (oracle) on the GPU's own
    profiles and greedy choice; a reload with other values replays correctly."""
    s = synth.four_regimes(per_regime=768)
    ms = [48, 64, 96, 128]
    K = 3
    from paper_2401_13680_b300 import pastila
    with _series(s.T, 0) as h:
        runs = [h.select_length(ms, K) for _ in range(3)]
        for r in runs[1:]:
            assert r[0] == runs[0][0] and np.array_equal(r[1], runs[0][1]) and r[2] == runs[0][2]
        for i, m in enumerate(ms):
            D, _ = h.profiles(m)
            Dd = D.astype(np.float64)
            c, _ = oracle.greedy(Dd, K)
            assert runs[0][1][i] == pytest.approx(oracle.criterion(Dd, c), rel=1e-12)
        T2 = synth.six_regime_sweep(seed=5, n=s.T.shape[0], min_len=300).T
        h.reload(T2)
        got = [h.select_length(ms, K) for _ in range(3)]
    with _series(T2, 0) as h2:
        fresh = h2.select_length(ms, K)
    for g in got:
        assert g[0] == fresh[0] and np.array_equal(g[1], fresh[1]) and g[2] == fresh[2]


def test_large_drift_series_full_size_sampled(lib):
    """n = 1,000,000 (eight regimes on a random-walk drift), m = 256, ell = 128,
    FP32, the whole S x P = 3,906 x 999,745 profile set (15.6 GB) resident on the
    device: 32 seeded segments x 4 seeded blocks of 256 positions checked cell by
    cell against the oracle's PSF steps, every value in [0, 2 sqrt(ell)], each
    sampled segment zero at its own offset, and D_max equal to the maximum of D;
    then the greedy snippets (K = 6) of the same profile set."""
    import torch
    from paper_2401_13680_b300 import pastila
    s = synth.large_drift()
    m, ell, k, K = 256, 128, 26, 6
    n = s.T.shape[0]
    S, P = n // m, n - m + 1
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(2024)
    segs = np.sort(rng.choice(S, 32, replace=False))
    blocks = rng.integers(0, P - 256, 4)
    with _series(s.T, 0) as h:
        D = torch.empty((S, P), dtype=torch.float32, device=dev)
        dmax = torch.zeros(1, dtype=torch.float64, device=dev)
        h.profiles_device(m, D.data_ptr(), dmax.data_ptr())
        torch.cuda.synchronize()
        assert float(D.min()) >= 0.0 and float(D.max()) <= 2 * np.sqrt(ell) * (1 + 1e-6)
        assert float(dmax.item()) == pytest.approx(float(D.max()), rel=1e-7)
        Ds = D[torch.from_numpy(segs).to(dev)]
        for b in blocks:
            ref = oracle.profiles_range(s.T, m, ell, k, segs, int(b), int(b) + 256)
            got = Ds[:, int(b):int(b) + 256].cpu().numpy()
            assert_profiles_close(got, ref, ell, TOL[0])
        own = Ds.cpu().numpy()[np.arange(32), segs * m]
        assert np.all(own == 0.0)
        del D, Ds
        torch.cuda.empty_cache()
        recs, _, _ = h.snippets(m, K)
    assert len({r[0] for r in recs}) == K
    assert sum(r[2] for r in recs) == pytest.approx(1.0)


def _purity(s, m, recs, labels):
    """Share of the positions whose window lies inside one planted regime that
    are labelled with a snippet from that regime, over the regimes that hold a
    snippet; a snippet belongs to the regime of its middle point (segments may
    straddle a regime boundary)."""
    snip_regime = {r[0]: s.regime_of(r[0] * m + m // 2) for r in recs}
    P = s.T.shape[0] - m + 1
    truth = np.array([s.regime_of(p) for p in range(P)])
    inside = truth == np.array([s.regime_of(p + m - 1) for p in range(P)])
    covered = np.isin(truth, list(set(snip_regime.values())))
    got = np.array([snip_regime[int(l)] for l in labels])
    sel = inside & covered
    return set(snip_regime.values()), float(np.mean(got[sel] == truth[sel]))


@pytest.mark.parametrize("prec", [0, 1])
def test_planted_regimes_recovered_and_labels_pure(lib, prec):
    """Four planted regimes, K = 4 (m = 128): the greedy snippets fall in the four
    regimes and the eq. 6 neighbour labels segment the series (label purity)."""
    s = synth.four_regimes()
    with _series(s.T, prec) as h:
        recs, labels, _ = h.snippets(128, 4, want_labels=True)
    regimes, purity = _purity(s, 128, recs, labels)
    assert regimes == {0, 1, 2, 3}
    assert purity >= 0.9, purity


def test_six_regime_labels(lib):
    """The six-regime sweep series, m = 256, K = 6 (FP32): the chirp, whose
    frequency drifts across its regime, takes two snippets, so five of the six
    regimes hold one (the AR(1) noise, which repeats no pattern, is labelled by
    its nearest neighbours); the labels follow the planted regimes."""
    s = synth.six_regime_sweep()
    with _series(s.T, 0) as h:
        recs, labels, _ = h.snippets(256, 6, want_labels=True)
    regimes, purity = _purity(s, 256, recs, labels)
    print("six-regime snippets in regimes", sorted(regimes), "label purity", purity)
    assert len(regimes) >= 5
    assert purity >= 0.9, purity
