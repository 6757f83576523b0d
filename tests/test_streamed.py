"""The greedy snippet search without the profile set (pastila_snippets_streamed
and the automatic switch to it in pastila_snippets): the same records, labels
and chosen profiles as the search on the materialised D, bit for bit (the
same tile layout, cluster tiles included; both decide every step on the
handle's own precision, so the FP32 comparison turns off the FP64 decision of
near-tied steps), with one full pass over the segments and few recomputed rows
where the area bounds prune, and a further pass at a step where they leave
more than half of the segments open.  On FP64 handles the streamed search also
equals the FP64 oracle."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _both(pastila, T, m, K, prec, budget=0):
    with pastila.Series(T, precision=prec) as h:
        h.set_fp64_ties(False)
        ref = h.snippets(m, K, want_labels=True, want_profiles=True)
    with pastila.Series(T, precision=prec, mem_budget=budget) as h:
        got = h.snippets_streamed(m, K, want_labels=True, want_profiles=True)
    return ref, got


def _same(ref, got):
    assert got[0] == ref[0]                      # records: index, rank, frac, area_after
    np.testing.assert_array_equal(got[1], ref[1])  # labels
    np.testing.assert_array_equal(got[2], ref[2])  # chosen profiles, greedy order


@pytest.mark.parametrize("prec", [0, 1])
def test_streamed_equals_materialised(lib, prec):
    from paper_2401_13680_b300 import pastila
    cases = [(synth.four_regimes().T, 128, 4), (synth.four_regimes().T, 96, 1),
             (synth.random_planted(np.random.default_rng(3), 20_000, 5).T, 160, 6)]
    if prec == 0:
        cases.append((synth.six_regime_sweep().T, 256, 6))
    for T, m, K in cases:
        ref, got = _both(pastila, T, m, K, prec)
        _same(ref, got)
        passes, rows = got[3]
        assert 1 <= passes <= K
        assert rows >= K
        S = T.shape[0] // m
        assert rows <= K * S  # never more than the materialised search's rows


def test_streamed_fp64_equals_the_oracle(lib):
    """FP64 handles: the streamed search's snippets, labels and areas are the
    oracle's (four regimes; a 20,000-point planted series)."""
    import oracle
    from paper_2401_13680_b300 import pastila
    cases = [(synth.four_regimes().T, 128, 4),
             (synth.random_planted(np.random.default_rng(3), 20_000, 5).T, 160, 6)]
    for T, m, K in cases:
        ell, k = m // 2, (m + 9) // 10
        chosen, area, labels, frac, order, D = oracle.snippets(T, m, ell, k, K)
        with pastila.Series(T, precision=1) as h:
            recs, lab, prof, _ = h.snippets_streamed(m, K, want_labels=True, want_profiles=True)
        assert [r[0] for r in recs] == [int(chosen[o]) for o in order]
        assert [r[1] for r in recs] == [int(o) for o in order]
        np.testing.assert_allclose([r[2] for r in recs], [frac[o] for o in order], rtol=0, atol=1e-12)
        np.testing.assert_allclose([r[3] for r in recs], [area[o] for o in order], rtol=1e-9)
        assert np.array_equal(lab, labels)
        np.testing.assert_allclose(prof, D[chosen], rtol=1e-9, atol=1e-9)


def test_streamed_exact_ties(lib):
    """A periodic series whose period divides m: every segment has the same
    profile, all areas tie exactly at every step, and the lowest index wins."""
    from paper_2401_13680_b300 import pastila
    base = synth.white_noise(7, 64)
    T = np.tile(base, 60)
    ref, got = _both(pastila, T, 128, 3, 0)
    _same(ref, got)
    assert [r[0] for r in sorted(got[0], key=lambda r: r[1])] == [0, 1, 2]
    # no bound can separate equal areas: steps 1 and 2 fall back to a pass
    assert got[3][0] == 3


def test_snippets_switches_to_streaming_when_d_does_not_fit(lib):
    from paper_2401_13680_b300 import pastila
    s = synth.six_regime_sweep()
    m, K = 256, 4
    S, P = s.T.shape[0] // m, s.T.shape[0] - m + 1
    d_bytes = 4 * S * P
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        h.set_fp64_ties(False)
        ref = h.snippets(m, K, want_labels=True, want_profiles=True)
    budget = d_bytes // 4  # far too small for D, enough for the streamed search
    with pastila.Series(s.T, precision=pastila.FP32, mem_budget=budget) as h:
        got = h.snippets(m, K, want_labels=True, want_profiles=True)
        with pytest.raises(pastila.PastilaError, match="ENOMEM"):
            h.profiles(m)  # the profile set itself still cannot be produced
    _same(ref, got)


def test_streamed_on_ecg_like_series(lib):
    """The stress workload's kind of series (ECG-like beats, morphology regimes)
    at n = 200,000, m = 256, K = 8: streamed equals materialised."""
    from paper_2401_13680_b300 import pastila
    s = synth.ecg_like(n=200_000)
    ref, got = _both(pastila, s.T, 256, 8, 0)
    _same(ref, got)


def test_streamed_with_cluster_tiles(lib):
    """With a two-CTA cluster layout in force the streamed search uses it too,
    and its results stay those of the materialised search."""
    from paper_2401_13680_b300 import pastila
    rng = np.random.default_rng(8)
    T = synth.random_planted(rng, 30_000, 5).T
    m, K = 256, 5
    pastila.tune_clear()
    try:
        pastila.tune_set(pastila.FP32, m, m // 2, (m + 9) // 10, 256, 2, 32, 2)
        with pastila.Series(T, precision=pastila.FP32) as h:
            assert h.tile_layout(m)["CS"] == 2
        ref, got = _both(pastila, T, m, K, 0)
        _same(ref, got)
    finally:
        pastila.tune_clear()
