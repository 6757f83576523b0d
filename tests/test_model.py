"""The runtime model (pastila_model_*): a polynomial regression of device time
on the work of a sweep, in the spirit of the run-time prediction of Section
4.2.  Host code only: these tests feed it observations whose times follow
known coefficients and check what it recovers, its warm start, its reset and
its argument checks.  No call here reaches a device."""
import numpy as np
import pytest

from paper_2401_13680_b300 import pastila

SMEM = 232448 - 1024


@pytest.fixture()
def fresh_model():
    """Each test starts from the prior and leaves the process-wide models as it found them."""
    saved = {p: pastila.model_get(p) for p in (pastila.FP32, pastila.FP64)}
    for p in saved:
        pastila.model_reset(p)
    yield
    for p, m in saved.items():
        pastila.model_set(m)


def _features(rng, n_chunks):
    """Features of a wave of n_chunks tile chunks at random lengths, plus greedy reads."""
    f = np.zeros(5)
    for _ in range(n_chunks):
        E = rng.uniform(0.05, 3.0)          # 1e9 cells
        x = rng.choice(np.arange(64, 769, 32)) / 256.0
        f[:3] += E * np.array([1.0, x, x * x])
    f[3] = rng.choice([0.0, rng.uniform(0.1, 40.0)])
    f[4] = 1.0
    return f


TRUE = np.array([9.0, 1.5, -0.4, 0.3, 0.07])


def test_recovers_known_coefficients(fresh_model):
    rng = np.random.default_rng(0)
    obs = [_features(rng, int(rng.integers(1, 6))) for _ in range(60)]
    for f in obs:
        pastila.model_observe(pastila.FP32, f, float(f @ TRUE))
    m = pastila.model_get(pastila.FP32)
    assert m["observations"] == 60
    np.testing.assert_allclose(m["coef"], TRUE, rtol=0.05, atol=0.02)  # the ridge biases collinear directions a little
    # held-out waves are predicted to well under a percent
    for _ in range(20):
        f = _features(rng, int(rng.integers(1, 6)))
        pred = f @ m["coef"]
        assert abs(pred - f @ TRUE) <= 5e-3 * (f @ TRUE)
    # the error bookkeeping counts the predictions made after 8 observations
    assert m["err_count"] == 60 - 8
    assert 0.0 <= m["rel_err"] < 0.2
    # the FP64 model is untouched
    assert pastila.model_get(pastila.FP64)["observations"] == 0


def test_cost_per_cell_follows_a_quadratic_in_m(fresh_model):
    # single-length observations: the fitted c0 + c1 x + c2 x^2 is the time per
    # 1e9 cells at each length
    rng = np.random.default_rng(1)
    for _ in range(40):
        m = int(rng.choice(np.arange(64, 769, 32)))
        x = m / 256.0
        E = rng.uniform(0.5, 4.0)
        f = np.array([E, E * x, E * x * x, 0.0, 1.0])
        pastila.model_observe(pastila.FP32, f, float(f @ TRUE))
    c = pastila.model_get(pastila.FP32)["coef"]
    for m in (64, 256, 512, 768):
        x = m / 256.0
        per = c[0] + c[1] * x + c[2] * x * x
        assert abs(per - (TRUE[0] + TRUE[1] * x + TRUE[2] * x * x)) < 0.02 * TRUE[0]


def test_collinear_data_keeps_the_prior_where_it_says_nothing(fresh_model):
    # every wave at m = 256 with no greedy reads: the model learns the rate at
    # x = 1 and the per-wave cost; the greedy coefficient stays at its prior
    prior = pastila.model_get(pastila.FP32)["prior"]
    for E in np.linspace(0.5, 4.0, 30):
        f = np.array([E, E, E, 0.0, 1.0])
        pastila.model_observe(pastila.FP32, f, float(12.0 * E + 0.1))
    m = pastila.model_get(pastila.FP32)
    assert np.all(np.isfinite(m["coef"]))
    assert abs(m["coef"][:3].sum() - 12.0) < 0.05
    assert m["coef"][3] == pytest.approx(prior[3], rel=1e-6)
    f = np.array([2.0, 2.0, 2.0, 0.0, 1.0])
    assert f @ m["coef"] == pytest.approx(24.1, rel=5e-3)


def test_warm_start_round_trip_and_reset(fresh_model):
    rng = np.random.default_rng(2)
    for _ in range(25):
        f = _features(rng, 3)
        pastila.model_observe(pastila.FP64, f, float(f @ (TRUE * 12)))
    saved = pastila.model_get(pastila.FP64)
    pastila.model_reset(pastila.FP64)
    cleared = pastila.model_get(pastila.FP64)
    assert cleared["observations"] == 0
    np.testing.assert_array_equal(cleared["coef"], cleared["prior"])
    pastila.model_set(saved)
    back = pastila.model_get(pastila.FP64)
    np.testing.assert_array_equal(back["coef"], saved["coef"])
    np.testing.assert_array_equal(back["xtx"], saved["xtx"])
    assert back["observations"] == saved["observations"]


def test_job_prediction(fresh_model):
    ms = [64, 128, 256]
    small = pastila.model_predict(pastila.FP32, 20_000, ms, 3, SMEM)
    large = pastila.model_predict(pastila.FP32, 200_000, ms, 3, SMEM)
    assert 0 < small < large
    # the tile work grows about as n^2: so does the prediction (prior: 11 ms per 1e9 cells)
    assert 60 < large / small < 140
    # FP64 is predicted slower than FP32 (its prior rate)
    assert pastila.model_predict(pastila.FP64, 20_000, ms, 3, SMEM) > small
    # n = 1e5, m = 256: S = 390 segments, 129 rows, about 1e5 columns (plus halo)
    p = pastila.model_predict(pastila.FP32, 100_000, [256], 4, SMEM)
    cells = 390 * 129 * 99_745
    assert 11.0 * cells * 1e-9 < p < 11.0 * 3.0 * cells * 1e-9


def test_argument_errors(fresh_model):
    with pytest.raises(pastila.PastilaError, match="EINVAL"):
        pastila.model_observe(pastila.FP32, [1, 1, 1, 0, 1], 0.0)
    with pytest.raises(pastila.PastilaError, match="EINVAL"):
        pastila.model_observe(pastila.FP32, [np.nan, 1, 1, 0, 1], 1.0)
    with pytest.raises(pastila.PastilaError, match="EINVAL"):
        pastila.model_observe(7, [1, 1, 1, 0, 1], 1.0)
    bad = pastila.model_get(pastila.FP32)
    bad["n_coef"] = 4
    with pytest.raises(pastila.PastilaError, match="n_coef"):
        pastila.model_set(bad)
    bad = pastila.model_get(pastila.FP32)
    bad["xtx"][0, 0] = np.inf
    with pytest.raises(pastila.PastilaError, match="finite"):
        pastila.model_set(bad)
    with pytest.raises(pastila.PastilaError, match="K = 1"):
        pastila.model_predict(pastila.FP32, 20_000, [64], 1, SMEM)
    with pytest.raises(pastila.PastilaError, match="n_m"):
        pastila.model_predict(pastila.FP32, 20_000, [], 3, SMEM)
