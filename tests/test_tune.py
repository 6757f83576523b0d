"""The tile-layout autotuner (pastila_tune): it keeps a layout at least as fast
as the cost model's on its sample, the tuned layout still meets the oracle
tolerance, a layout always gives the same results, and a captured
select_length graph follows a change of layout."""
import numpy as np
import pytest

import oracle
import synth
from tolerance import assert_profiles_close

pytestmark = pytest.mark.gpu


@pytest.fixture
def clean_table(lib):
    from paper_2401_13680_b300 import pastila
    pastila.tune_clear()
    yield pastila
    pastila.tune_clear()


def test_tuned_layouts_are_faster_and_within_tolerance(clean_table):
    pastila = clean_table
    s = synth.four_regimes()
    ms = [64, 128, 256]
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        before = {m: h.profiles(m)[0] for m in ms}
        res = h.tune(ms, max_candidates=6)
        after = {m: h.profiles(m)[0] for m in ms}
        again = {m: h.profiles(m)[0] for m in ms}
    for r in res:
        assert r["candidates"] >= 1 and r["ms_best"] <= r["ms_model"] + 1e-9
        assert r["NT"] <= 512 and r["W"] % 32 == 0
    for m in ms:
        np.testing.assert_array_equal(after[m], again[m])  # one layout, one result
        ref = oracle.profiles(s.T, m, m // 2, (m + 9) // 10)
        assert_profiles_close(after[m], ref, m // 2, 1e-4)
    pastila.tune_clear()
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        for m in ms:  # the cost model's layout again: the first results exactly
            np.testing.assert_array_equal(h.profiles(m)[0], before[m])


def test_captured_graph_follows_a_new_layout(clean_table):
    pastila = clean_table
    s = synth.four_regimes()
    ms, K = [96, 128, 160], 3
    with pastila.Series(s.T, precision=pastila.FP32) as h:
        for _ in range(3):  # the second call captures, the third replays
            first = h.select_length(ms, K)
        h.tune(ms, max_candidates=4)
        tuned = h.select_length(ms, K)  # rebuilt for the tuned layouts
        tuned2 = h.select_length(ms, K)
        tuned3 = h.select_length(ms, K)  # replay of the new capture
    with pastila.Series(s.T, precision=pastila.FP32) as h2:
        fresh = h2.select_length(ms, K)
    for r in (tuned2, tuned3, fresh):
        assert r[0] == tuned[0]
        np.testing.assert_array_equal(r[1], tuned[1])
        assert r[2] == tuned[2]
    # a layout change moves the criterion by FP32 rounding only
    np.testing.assert_allclose(tuned[1], first[1], rtol=1e-4)


def test_tune_argument_errors(lib):
    from paper_2401_13680_b300 import pastila
    with pastila.Series(synth.white_noise(1, 3000), precision=pastila.FP32) as h:
        with pytest.raises(pastila.PastilaError, match="max_candidates"):
            h.tune([64], max_candidates=0)
        with pytest.raises(pastila.PastilaError, match="exceeds"):
            h.tune([5000])
