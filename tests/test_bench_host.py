"""Host logic of bench.py (no device): the cell counts behind the metric, the
first-come-first-served latency model of the serving leg's FP64 comparison,
and the multivariate leg's bookkeeping, the last with a stand-in for the
binding."""
import types

import numpy as np

import bench
import synth


def test_cell_counts_match_their_definitions():
    """Profile cells: S x P per length (S = floor(n / m) segments, P = n - m + 1
    positions); ED cells: S x R x C with R = m - ell + 1 row windows and
    C = n - ell + 1 column windows, ell = m / 2."""
    for n, ms in ((1000, [8, 12, 50]), (4096, [64, 96]), (100_000, synth.sweep_lengths())):
        prof = ed = 0
        for m in ms:
            ell = synth.default_ell(m)
            S, P, R, C = n // m, n - m + 1, m - ell + 1, n - ell + 1
            prof += S * P
            ed += S * R * C
        assert bench.cells(n, ms) == (prof, ed)
    job = types.SimpleNamespace(n=5000, ms=[64, 160])
    assert bench.job_profile_cells(job) == bench.cells(5000, [64, 160])[0]
    assert bench.job_ed_cells(job) == bench.cells(5000, [64, 160])[1]


def test_fifo_latencies_by_hand():
    # arrivals 0, 1, 10; service 2, 2, 1: the second waits for the first
    assert bench.fifo_latencies([0.0, 1.0, 10.0], [2.0, 2.0, 1.0]) == [2.0, 3.0, 1.0]
    assert bench.fifo_latencies([], []) == []


class _Engine:
    def __init__(self, results, device=0):
        self.results = results

    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass

    def submit_multivariate(self, T, ms, K):
        assert T.ndim == 2 and T.shape[0] == 3
        return list(range(T.shape[0]))

    def wait(self, j):
        return {"state": 3, "first_wave": 7}

    def result(self, j):
        return self.results[j]


class _Series:
    def __init__(self, results, T, device=0, precision=0):
        self.r = results[_Series.calls % 3]
        _Series.calls += 1

    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass

    def select_length(self, ms, K):
        return self.r


def _stub(engine_results, series_results):
    _Series.calls = 0
    return types.SimpleNamespace(
        Engine=lambda device=0: _Engine(engine_results, device),
        Series=lambda T, device=0, precision=0: _Series(series_results, T, device, precision),
        FP32=0, JOB_DONE=3)


def test_multivariate_leg_compares_every_coordinate():
    ms = [64, 128]
    res = [(64 + 64 * (c % 2), np.array([1.0 + c, 2.0]), [(c, 0, 0.5, 1.0)]) for c in range(3)]
    out = bench.run_multivariate(_stub(res, res), 0, ms, 2)
    assert out["results_identical"] and out["engine_first_waves"] == 1 and out["coordinates"] == 3
    assert out["engine_profile_cells_per_s"] > 0 and out["sequential_profile_cells_per_s"] > 0
    # one coordinate's record differs: the leg says so
    other = list(res)
    other[2] = (res[2][0], res[2][1], [(5, 0, 0.5, 1.0)])
    assert not bench.run_multivariate(_stub(res, other), 0, ms, 2)["results_identical"]
    # a criterion value differs
    other[2] = (res[2][0], res[2][1] + 1e-12, res[2][2])
    assert not bench.run_multivariate(_stub(res, other), 0, ms, 2)["results_identical"]


def test_error_ratio_follows_the_tolerance_rule():
    """Above d_floor = 0.1 sqrt(2 ell) the ratio is relative; below, |d^2 -
    d_ref^2| / (2 d_floor^2); the two agree at the floor (continuity)."""
    ell = 50
    fl = bench.d_floor(ell)
    assert fl == np.sqrt(100.0) * 0.1
    r = bench.profile_error_ratio([2.2, 0.0], [2.0, 0.5], ell)
    assert r[0] == np.abs(2.2 - 2.0) / 2.0
    assert r[1] == 0.25 / (2.0 * fl ** 2)
    eps = 1e-6
    above = bench.profile_error_ratio([fl * (1 + eps)], [fl], ell)[0]
    below = bench.profile_error_ratio([fl * (1 - 1e-12) * (1 + eps)], [fl * (1 - 1e-12)], ell)[0]
    assert abs(above - below) < 1e-9


def test_sample_cells_cover_tile_boundaries():
    """Every sampled cell is in range; the sample holds the first and last
    position and both sides of the first tile boundaries."""
    rng = np.random.default_rng(0)
    S, P, W = 300, 99_000, 480
    segs, pos = bench.sample_cells(S, P, W, 24, rng)
    assert segs.shape == pos.shape
    assert segs.min() >= 0 and segs.max() < S and pos.min() >= 0 and pos.max() < P
    got = set(pos.tolist())
    assert {0, P - 1, W - 1, W, 2 * W - 1, 2 * W} <= got
    assert 0 in segs.tolist() and S - 1 in segs.tolist()


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    """The recorded DRAM traffic counts only while the kernel sources hash to the
    value the capture recorded."""
    import json
    f = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic()[0] is None  # no file
    f.write_text(json.dumps({"kernel_sources_sha256": bench.tile_sources_sha(),
                             "dram_bytes_per_sweep_step": 3.0e9, "capture": "ncu ..."}))
    assert bench.measured_traffic() == (3.0e9, "ncu ...")
    f.write_text(json.dumps({"kernel_sources_sha256": "0" * 64, "dram_bytes_per_sweep_step": 3.0e9}))
    v, why = bench.measured_traffic()
    assert v is None and "predates" in why
