"""Seeded synthetic series shaped like the paper's labelling workloads.

The paper evaluates on TSSB, a solar-power series and PAMAP (Section 5.1.1);
none of them ships here, so these generators stand in for them with
planted-regime series of the same kind (several activities, each a repeated
pattern, plus noise).  This module holds no MPdist arithmetic: it only draws
inputs, and both the CUDA path and the CPU oracle consume what it returns.

Every series is float64, little-endian, contiguous; every draw comes from
``numpy.random.default_rng(seed)`` (PCG64), so the same seed gives the same
bytes on every machine.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# ----------------------------------------------------------------------------
# regime shapes: amplitude about 1, phase restarting at the regime start
# ----------------------------------------------------------------------------


def _sine(length: int, period: float) -> np.ndarray:
    i = np.arange(length, dtype=np.float64)
    return np.sin(2.0 * np.pi * i / period)


def _square(length: int, period: int) -> np.ndarray:
    # +1 on the first half-period, -1 on the second
    i = np.arange(length)
    return np.where((i % period) < (period // 2), 1.0, -1.0)


def _sawtooth(length: int, period: int) -> np.ndarray:
    i = np.arange(length)
    return 2.0 * (i % period) / period - 1.0


def _bumps(length: int, spacing: int, width: float = 5.0) -> np.ndarray:
    # Gaussian bumps centred at spacing/2 + q*spacing
    i = np.arange(length, dtype=np.float64)
    out = np.zeros(length)
    c = spacing / 2.0
    while c < length + 4 * width:
        out += np.exp(-0.5 * ((i - c) / width) ** 2)
        c += spacing
    return out


def _chirp(length: int, f0: float = 1.0 / 80, f1: float = 1.0 / 20) -> np.ndarray:
    # instantaneous frequency rises linearly from f0 to f1 over the regime
    i = np.arange(length, dtype=np.float64)
    f = f0 + (f1 - f0) * i / max(length - 1, 1)
    phase = 2.0 * np.pi * np.cumsum(f)
    return np.sin(phase - phase[0])


def _ar1(length: int, rng: np.random.Generator, phi: float = 0.9) -> np.ndarray:
    # unit-variance AR(1): innovations N(0, 1 - phi^2)
    e = rng.normal(0.0, np.sqrt(1.0 - phi * phi), size=length)
    out = np.empty(length)
    acc = rng.normal()
    for t in range(length):
        acc = phi * acc + e[t]
        out[t] = acc
    return out


REGIME_TYPES = ("sine", "square", "sawtooth", "bump", "chirp", "ar1")


def _regime(kind: str, length: int, period: float, rng: np.random.Generator) -> np.ndarray:
    if kind == "sine":
        return _sine(length, period)
    if kind == "square":
        return _square(length, int(round(period)))
    if kind == "sawtooth":
        return _sawtooth(length, int(round(period)))
    if kind == "bump":
        return _bumps(length, int(round(period)))
    if kind == "chirp":
        return _chirp(length)
    if kind == "ar1":
        return _ar1(length, rng)
    raise ValueError(kind)


@dataclasses.dataclass
class Series:
    """A synthetic series with its planted ground truth."""

    T: np.ndarray                 # float64 values
    bounds: list                  # [(start, stop, kind)] of each planted regime
    name: str

    def regime_of(self, i: int) -> int:
        for q, (a, b, _) in enumerate(self.bounds):
            if a <= i < b:
                return q
        return len(self.bounds) - 1


def _assemble(kinds, lengths, periods, rng, noise_sd, name):
    parts, bounds, start = [], [], 0
    for kind, ln, per in zip(kinds, lengths, periods):
        parts.append(_regime(kind, int(ln), per, rng))
        bounds.append((start, start + int(ln), kind))
        start += int(ln)
    T = np.concatenate(parts)
    if noise_sd > 0:
        T = T + rng.normal(0.0, noise_sd, size=T.shape[0])
    return Series(np.ascontiguousarray(T, dtype=np.float64), bounds, name)


# ----------------------------------------------------------------------------
# the workload recipes (sizes, seeds and parameters are the documented ones)
# ----------------------------------------------------------------------------


def four_regimes(seed: int = 0, per_regime: int = 1024, noise_sd: float = 0.1) -> Series:
    """n = 4 x 1024: sine (period 50), square (64), sawtooth (40), bumps every 80,
    in that order, plus N(0, 0.1^2) noise."""
    rng = np.random.default_rng(seed)
    kinds = ("sine", "square", "sawtooth", "bump")
    periods = (50, 64, 40, 80)
    return _assemble(kinds, [per_regime] * 4, periods, rng, noise_sd, "four_regimes_n4096")


def six_regime_sweep(seed: int = 1, n: int = 100_000, min_len: int = 5000,
                     noise_sd: float = 0.05) -> Series:
    """n = 100,000: six regimes (sine, square, sawtooth, bump, chirp, AR(1) phi=0.9)
    in random order, lengths min_len + Dirichlet(1,...,1)*(n - 6*min_len),
    plus N(0, 0.05^2) noise."""
    rng = np.random.default_rng(seed)
    kinds = list(REGIME_TYPES)
    order = rng.permutation(len(kinds))
    kinds = [kinds[q] for q in order]
    w = rng.dirichlet(np.ones(len(kinds)))
    free = n - len(kinds) * min_len
    lengths = (min_len + np.floor(w * free)).astype(np.int64)
    lengths[-1] = n - lengths[:-1].sum()
    base_period = {"sine": 50, "square": 64, "sawtooth": 40, "bump": 80, "chirp": 0, "ar1": 0}
    periods = [base_period[k] for k in kinds]
    return _assemble(kinds, lengths, periods, rng, noise_sd, "six_regime_sweep_n100000")


def large_drift(seed: int = 2, n: int = 1_000_000, n_regimes: int = 8,
                drift_sd: float = 0.01) -> Series:
    """n = 1,000,000: 8 regimes with lengths U[50k, 250k] rescaled to sum n, kinds
    drawn from the six-regime set, periodic kinds with period U[30, 120];
    plus a random-walk drift cumsum(N(0, 0.01^2)) and no white noise."""
    rng = np.random.default_rng(seed)
    raw = rng.uniform(50_000, 250_000, size=n_regimes)
    lengths = np.floor(raw / raw.sum() * n).astype(np.int64)
    lengths[-1] = n - lengths[:-1].sum()
    kinds = [REGIME_TYPES[q] for q in rng.integers(0, len(REGIME_TYPES), size=n_regimes)]
    periods = rng.uniform(30, 120, size=n_regimes)
    s = _assemble(kinds, lengths, periods, rng, 0.0, "large_drift_n1000000")
    s.T = np.ascontiguousarray(s.T + np.cumsum(rng.normal(0.0, drift_sd, size=n)))
    return s


def random_planted(rng: np.random.Generator, n: int, n_regimes: int, noise_sd: float = 0.05,
                   name: str = "planted") -> Series:
    """A series of length n from n_regimes random kinds with random periods in
    [30, 120] and random lengths (each at least n / (4 n_regimes))."""
    kinds = [REGIME_TYPES[q] for q in rng.integers(0, len(REGIME_TYPES), size=n_regimes)]
    w = rng.dirichlet(np.ones(n_regimes))
    min_len = n // (4 * n_regimes)
    lengths = (min_len + np.floor(w * (n - n_regimes * min_len))).astype(np.int64)
    lengths[-1] = n - lengths[:-1].sum()
    periods = rng.uniform(30, 120, size=n_regimes)
    return _assemble(kinds, lengths, periods, rng, noise_sd, name)


def sweep_lengths(lo: int = 64, hi: int = 512, step: int = 32) -> list:
    """The snippet lengths m of the six-regime sweep: 64, 96, ..., 512."""
    return list(range(lo, hi + 1, step))


def default_ell(m: int) -> int:
    """Inner subsequence length used by every workload here: ell = m / 2."""
    return m // 2


def default_k(m: int) -> int:
    """MPdist rank: ceil(0.05 * 2m) in integer arithmetic, i.e. (m + 9) // 10."""
    return (m + 9) // 10


def white_noise(seed: int, n: int, sd: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).normal(0.0, sd, size=n)


# ----------------------------------------------------------------------------
# serving workload: a stream of independent labelling jobs
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Job:
    """One serving job: a planted-regime series and its own length sweep."""

    arrival: float      # seconds after the first arrival
    n: int
    ms: list            # distinct snippet lengths, ascending
    K: int
    n_regimes: int
    seed: int           # seed of the series' generator

    def series(self) -> np.ndarray:
        rng = np.random.default_rng(self.seed)
        return random_planted(rng, self.n, self.n_regimes, 0.05, name=f"job_n{self.n}").T


def serving_jobs(n_jobs: int = 1000, rate: float = 20.0, seed: int = 3, n_lo: int = 10_000,
                 n_hi: int = 500_000) -> list:
    """Poisson arrivals at `rate` jobs/s (exponential gaps, first job at t = 0);
    n log-uniform in [n_lo, n_hi]; 3-8 planted regimes from the six-regime set
    plus N(0, 0.05^2) noise; a sweep of 3-10 distinct lengths from the multiples
    of 32 in [64, 768]; ell = m / 2; K uniform in [3, 6]."""
    rng = np.random.default_rng(seed)
    grid = np.arange(64, 769, 32)
    jobs, t = [], 0.0
    for q in range(n_jobs):
        if q:
            t += float(rng.exponential(1.0 / rate))
        n = int(round(float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))))
        n_m = int(rng.integers(3, 11))
        ms = sorted(int(x) for x in rng.choice(grid, size=n_m, replace=False))
        K = int(rng.integers(3, 7))
        n_reg = int(rng.integers(3, 9))
        jobs.append(Job(t, n, ms, K, n_reg, int(rng.integers(0, 2**31 - 1))))
    return jobs


# ----------------------------------------------------------------------------
# ECG-like stress series
# ----------------------------------------------------------------------------

# PQRST beat template: five Gaussian waves (centre offset in samples from the R
# peak, width in samples, amplitude) at the RR scale of 800 samples
_PQRST = ((-200.0, 25.0, 0.12), (-45.0, 8.0, -0.10), (0.0, 10.0, 1.00), (40.0, 9.0, -0.25), (260.0, 45.0, 0.30))


def ecg_like(n: int = 10_000_000, seed: int = 4, n_regimes: int = 12, noise_sd: float = 0.02) -> Series:
    """n samples of beats at RR ~ N(800, 40) samples; n_regimes consecutive
    morphology regimes of equal length, each scaling every wave's amplitude by
    U[0.6, 1.4] and width by U[0.7, 1.3] (drawn once per regime); plus
    N(0, 0.02^2) noise."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.6, 1.4, size=(n_regimes, len(_PQRST)))
    wid = rng.uniform(0.7, 1.3, size=(n_regimes, len(_PQRST)))
    T = np.zeros(n)
    bounds, per = [], n // n_regimes
    for q in range(n_regimes):
        a, b = q * per, (n if q == n_regimes - 1 else (q + 1) * per)
        bounds.append((a, b, f"morphology{q}"))
    pos = 300.0
    while pos < n + 600:
        q = min(int(pos) // per, n_regimes - 1) if pos < n else n_regimes - 1
        lo, hi = max(0, int(pos) - 400), min(n, int(pos) + 500)
        if lo < hi:
            i = np.arange(lo, hi, dtype=np.float64)
            for w, (c, sd, A) in enumerate(_PQRST):
                s = sd * wid[q, w]
                T[lo:hi] += A * amp[q, w] * np.exp(-0.5 * ((i - pos - c) / s) ** 2)
        pos += rng.normal(800.0, 40.0)
    T += rng.normal(0.0, noise_sd, size=n)
    return Series(np.ascontiguousarray(T), bounds, f"ecg_like_n{n}")
