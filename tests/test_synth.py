"""The seeded input generators: shapes, layouts and the documented recipes
(sizes, regime counts and lengths, seeds, the serving stream's ranges); they
hold no MPdist arithmetic."""
import numpy as np

import synth


def test_ecg_like_generator_shape():
    """The ECG-like series has one R peak per RR interval (mean 800 samples) and
    its documented regime layout (inputs only; no MPdist arithmetic)."""
    s = synth.ecg_like(n=80_000, n_regimes=4)
    T = s.T
    from scipy.signal import find_peaks
    peaks, _ = find_peaks(T, height=0.5, distance=400)
    gaps = np.diff(peaks)
    assert 700 < gaps.mean() < 900
    assert [b[:2] for b in s.bounds] == [(0, 20000), (20000, 40000), (40000, 60000), (60000, 80000)]


def _contiguous(bounds, n):
    assert bounds[0][0] == 0 and bounds[-1][1] == n
    assert all(a[1] == b[0] for a, b in zip(bounds, bounds[1:]))
    return [b - a for a, b, _ in bounds]


def test_four_regimes_recipe():
    s = synth.four_regimes()
    assert s.T.shape == (4096,) and s.T.dtype == np.float64 and s.T.flags.c_contiguous
    assert s.bounds == [(0, 1024, "sine"), (1024, 2048, "square"), (2048, 3072, "sawtooth"), (3072, 4096, "bump")]
    assert np.array_equal(s.T, synth.four_regimes().T)          # same seed, same bytes
    assert not np.array_equal(s.T, synth.four_regimes(seed=9).T)


def test_six_regime_sweep_recipe():
    s = synth.six_regime_sweep()
    assert s.T.shape == (100_000,)
    lengths = _contiguous(s.bounds, 100_000)
    assert sorted(k for _, _, k in s.bounds) == sorted(synth.REGIME_TYPES) and len(lengths) == 6
    assert min(lengths) >= 5000
    assert np.array_equal(s.T, synth.six_regime_sweep().T)
    assert synth.sweep_lengths() == list(range(64, 513, 32))
    assert [synth.default_ell(m) for m in (64, 96, 512)] == [32, 48, 256]
    assert [synth.default_k(m) for m in (64, 96, 100, 512)] == [7, 10, 10, 52]  # ceil(0.1 m)


def test_large_drift_recipe():
    s = synth.large_drift()
    lengths = _contiguous(s.bounds, 1_000_000)
    assert len(lengths) == 8 and min(lengths) > 20_000
    assert {k for _, _, k in s.bounds} <= set(synth.REGIME_TYPES)


def test_random_planted_recipe():
    s = synth.random_planted(np.random.default_rng(5), 30_000, 5)
    lengths = _contiguous(s.bounds, 30_000)
    assert len(lengths) == 5 and min(lengths) >= 30_000 // 20


def test_serving_stream_recipe():
    jobs = synth.serving_jobs()
    assert len(jobs) == 1000 and jobs[0].arrival == 0.0
    arr = np.array([j.arrival for j in jobs])
    assert np.all(np.diff(arr) >= 0)
    assert 0.045 < np.diff(arr).mean() < 0.055                   # 20 jobs/s
    for j in jobs:
        assert 10_000 <= j.n <= 500_000 and 3 <= j.K <= 6 and 3 <= j.n_regimes <= 8
        assert 3 <= len(j.ms) <= 10 and j.ms == sorted(set(j.ms))
        assert all(64 <= m <= 768 and m % 32 == 0 for m in j.ms)
    assert [(j.n, j.ms) for j in synth.serving_jobs(n_jobs=32)] == [(j.n, j.ms) for j in jobs[:32]]
