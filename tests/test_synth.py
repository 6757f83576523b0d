"""The seeded input generators: shapes and layouts only (they hold no MPdist
arithmetic)."""
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
