"""Tiles computed by a thread-block cluster of two or four CTAs (each computes
its share of the rows of a wider tile and writes its row-window maxima for the
other CTAs' positions into their shared memory): parity with the oracle in
both precisions, a sweep mixing one-, two- and four-CTA tiles, the engine, and
the tuned-table entry points that force and report the layout."""
import numpy as np
import pytest

import oracle
import synth
from tolerance import assert_profiles_close

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-9}


@pytest.fixture
def table(lib):
    from paper_2401_13680_b300 import pastila
    pastila.tune_clear()
    yield pastila
    pastila.tune_clear()


def _force(pastila, prec, m, ell, k, W, NG, GS, CS=2):
    pastila.tune_set(prec, m, ell, k, W, NG, GS, CS)
    assert pastila.tune_get(prec, m, ell, k) == (W, NG, GS, CS)


# (n, m, ell, k, W, NG, GS, CS): R = 65, 101, 129 (rows held in 3-5 registers per
# lane) and 321 (beyond the register cache), with a ragged last tile and a tail segment
CLUSTER_CASES = [
    (4096, 128, 64, 13, 256, 2, 32, 2),
    (3001, 200, 100, 20, 192, 2, 32, 2),
    (5003, 256, 128, 26, 192, 3, 32, 2),
    (4000, 640, 320, 64, 64, 2, 32, 2),
    (5003, 256, 128, 26, 256, 2, 32, 4),
    (4000, 640, 320, 64, 128, 2, 32, 4),
]


@pytest.mark.parametrize("n,m,ell,k,W,NG,GS,CS", CLUSTER_CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_cluster_tiles_match_the_oracle(table, prec, n, m, ell, k, W, NG, GS, CS):
    pastila = table
    rng = np.random.default_rng(n + m)
    T = synth.random_planted(rng, n, 3).T if prec == 1 else np.cumsum(rng.normal(0, 0.2, n)) + rng.normal(0, 1.0, n)
    _force(pastila, prec, m, ell, k, W, NG, GS, CS)
    with pastila.Series(T, precision=prec) as h:
        lay = h.tile_layout(m, ell=ell, k=k)
        assert lay["CS"] == CS and lay["W"] == W, lay
        D, dmax = h.profiles(m, ell=ell, k=k)
    ref = oracle.profiles(T, m, ell, k)
    assert_profiles_close(D, ref, ell, TOL[prec])
    assert dmax == pytest.approx(float(D.max()), rel=1e-7)


def test_sweep_mixing_one_and_two_cta_tiles(table):
    """One sweep holds lengths with one-, two- and four-CTA tiles (one tile launch
    per cluster size); each criterion equals eq. 18 on the GPU's own profiles."""
    pastila = table
    s = synth.four_regimes(per_regime=750)  # n = 3000
    ms, K = [96, 128, 160, 192, 256], 3
    _force(pastila, 0, 96, 48, 10, 608, 1, 32, CS=1)
    _force(pastila, 0, 128, 64, 13, 192, 2, 32)
    _force(pastila, 0, 192, 96, 20, 160, 2, 32)
    _force(pastila, 0, 256, 128, 26, 256, 2, 32, CS=4)
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        assert [h.tile_layout(m)["CS"] for m in ms] == [1, 2, 1, 2, 4]
        runs = [h.select_length(ms, K) for _ in range(3)]  # direct, captured, replayed
        for r in runs[1:]:
            assert r[0] == runs[0][0] and np.array_equal(r[1], runs[0][1]) and r[2] == runs[0][2]
        for i, m in enumerate(ms):
            D, _ = h.profiles(m)
            Dd = D.astype(np.float64)
            c, _ = oracle.greedy(Dd, K)
            assert runs[0][1][i] == pytest.approx(oracle.criterion(Dd, c), rel=1e-12)
            ref = oracle.profiles(s.T, m, m // 2, (m + 9) // 10)
            assert_profiles_close(D, ref, m // 2, 1e-4)


def test_engine_with_cluster_tiles(table):
    pastila = table
    rng = np.random.default_rng(77)
    T = synth.random_planted(rng, 30_000, 4).T
    ms, K = [128, 160, 256, 384], 4
    _force(pastila, 0, 128, 64, 13, 256, 2, 32)
    _force(pastila, 0, 256, 128, 26, 192, 3, 32)
    _force(pastila, 0, 384, 192, 39, 384, 2, 32, CS=4)
    with pastila.Series(T, precision=pastila.FP32) as h:
        ref = h.select_length(ms, K)
    with pastila.Engine(wave_ed_cells=5e7) as e:
        j = e.submit(T, ms, K)
        assert e.wait(j)["state"] == pastila.JOB_DONE
        got = e.result(j)
    assert got[0] == ref[0]
    np.testing.assert_array_equal(got[1], ref[1])
    assert got[2] == ref[2]


def test_tune_set_argument_errors(lib):
    from paper_2401_13680_b300 import pastila
    with pytest.raises(pastila.PastilaError, match="CS = 3"):
        pastila.tune_set(0, 128, 64, 13, 256, 2, 32, 3)
    with pytest.raises(pastila.PastilaError, match="multiple of 32"):
        pastila.tune_set(0, 128, 64, 13, 250, 2, 32, 1)
    with pytest.raises(pastila.PastilaError, match="GS = 4: the selection runs one warp"):
        pastila.tune_set(0, 128, 64, 13, 256, 2, 4, 1)
    with pytest.raises(pastila.PastilaError, match="no tuned layout"):
        pastila.tune_get(0, 123, 61, 13)


def test_two_ctas_per_sm_layouts(table):
    """Layouts of at most 256 threads and half an SM's shared memory (two CTAs per
    SM) get a tile launch of their own in a sweep: parity with the oracle, one
    more tile launch than with the model's layouts, the same criterion as eq. 18
    on the GPU's own profiles, and the engine's results equal select_length."""
    pastila = table
    s = synth.four_regimes(per_regime=750)  # n = 3000
    ms, K = [64, 96, 128, 160], 3
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        h.select_length(ms, K)
        l0 = h.kernel_launches()
        h.select_length(ms, K)
        base_launches = h.kernel_launches() - l0
    _force(pastila, 0, 64, 32, 7, 480, 2, 32, CS=1)
    _force(pastila, 0, 128, 64, 13, 320, 2, 32, CS=1)
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        for m in (64, 128):
            lay = h.tile_layout(m)
            assert lay["NT"] <= 256 and lay["CS"] == 1, lay
        r = h.select_length(ms, K)
        l0 = h.kernel_launches()
        r2 = h.select_length(ms, K)
        assert h.kernel_launches() - l0 == base_launches + 1  # the two-CTA-per-SM launch
        assert r2[0] == r[0] and np.array_equal(r2[1], r[1])
        for i, m in enumerate(ms):
            D, _ = h.profiles(m)
            Dd = D.astype(np.float64)
            c, _ = oracle.greedy(Dd, K)
            assert r[1][i] == pytest.approx(oracle.criterion(Dd, c), rel=1e-12)
            ref = oracle.profiles(s.T, m, m // 2, (m + 9) // 10)
            assert_profiles_close(D, ref, m // 2, 1e-4)
    with pastila.Engine(wave_ed_cells=3e6) as e:
        j = e.submit(s.T, ms, K)
        assert e.wait(j)["state"] == pastila.JOB_DONE
        got = e.result(j)
    assert got[0] == r[0]
    np.testing.assert_array_equal(got[1], r[1])
    assert got[2] == r[2]
