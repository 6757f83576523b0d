"""The seeded input generators: shapes and layouts only (they hold no MPdist
arithmetic)."""
import numpy as np

import synth


def test_ecg_like_generator_shape():
    """The ECG-like series has one R peak per RR interval (mean 800 samples) and
    its documented regime layout (inputs only; no MPdist arithmetic)."""
    s = synth.ecg_like(n=80_000, n_regimes=4)
    T = s.T
    peaks = [i for i in range(1, T.shape[0] - 1)
             if T[i] > 0.5 and T[i] >= T[i - 1] and T[i] >= T[i + 1] and T[i] == T[max(0, i - 100):i + 100].max()]
    gaps = np.diff(peaks)
    assert 700 < gaps.mean() < 900
    assert [b[:2] for b in s.bounds] == [(0, 20000), (20000, 40000), (40000, 60000), (60000, 80000)]
