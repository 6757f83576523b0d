#!/usr/bin/env python
"""Benchmark of the MPdist-profile engine on the six-regime length sweep.

Workload (one "step" = the whole hot path once): a seeded six-regime series of
n = 100,000 points, snippet lengths m = 64, 96, ..., 512 (15 lengths), ell = m/2,
k = ceil(0.05 * 2m), K = 4 snippets: window statistics per ell, the profile set
D of every length, greedy snippets, neighbour shares and the length criterion,
ending in m_best -- one ``pastila_select_length`` call through the C ABI.

Metric: MPdist profile cells per second, a cell being one D_s(p) (sum over the
sweep of floor(n/m) * (n - m + 1) per step).  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A serving leg follows (``--serve-jobs``, 0 to skip): the first jobs of the
seeded serving stream (n log-uniform in [10^4, 5*10^5], 3-10 lengths in
[64, 768], K in [3, 6], Poisson arrivals) submitted in real time to the
serving engine, with the arrival clock scaled so that the offered load is
``--serve-load`` of the ED-cell rate the sweep leg measured; it reports p50/p99
job latency (arrival to results on the host) beside the engine's throughput,
and the p50/p99 that the plain FP64 one-job path would give on the same
arrivals (first come, first served, service times from its measured rate).

``--impl reference`` times the FP64 CPU oracle (the paper's definitions, PSF
steps) on a bounded sample of the same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

import synth  # noqa: E402

METRIC = "MPdist profile cells/s"
UNIT = "cells/s"
K_SNIPPETS = 4
SM_COUNT_B300 = 148
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2032.0
# algorithmic FP32 FLOPs per ED cell (eq. 9 matrix entry): 2 FMA of the covariance
# recurrence (4 FLOP), 2 multiplications by the inverse norms (2 FLOP), and the
# exact seed of every diagonal (ell FMA per R cells, about 2 FLOP at ell = m/2)
FLOP_PER_ED_CELL = 8.0
# DRAM traffic of one sweep step's tile launches: read from profiles/tile_traffic.json,
# an ncu capture of the kernel sources whose SHA-256 it records; reported only while
# those sources are unchanged (null otherwise)
TRAFFIC_FILE = os.path.join(HERE, "profiles", "tile_traffic.json")
TILE_SOURCES = [os.path.join(HERE, "paper_2401_13680_b300", "csrc", f) for f in ("tile.cuh", "batch.cuh", "keys.cuh")]


def tile_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in TILE_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_capture():
    """The recorded ncu figures of the tile kernel if they were taken on the current
    kernel sources: (record, None), else (None, why)."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None, "no recorded capture"
    if rec.get("kernel_sources_sha256") != tile_sources_sha():
        return None, "the recorded capture predates the current kernel sources"
    return rec, None


def measured_traffic():
    """(bytes per sweep step, provenance) from the recorded capture, or (None, why)."""
    rec, why = recorded_capture()
    if rec is None:
        return None, why
    return float(rec["dram_bytes_per_sweep_step"]), rec.get("capture", "")


def d_floor(ell):
    return 0.1 * np.sqrt(2.0 * ell)


def profile_error_ratio(d, d_ref, ell):
    """Per-cell error under the tolerance rule (relative above d_floor = 0.1 sqrt(2 ell),
    |d^2 - d_ref^2| / (2 d_floor^2) below it); compare with 1e-4 for FP32."""
    d = np.asarray(d, dtype=np.float64)
    d_ref = np.asarray(d_ref, dtype=np.float64)
    fl = d_floor(ell)
    above = d_ref >= fl
    r = np.empty_like(d_ref)
    r[above] = np.abs(d[above] - d_ref[above]) / d_ref[above]
    r[~above] = np.abs(d[~above] ** 2 - d_ref[~above] ** 2) / (2.0 * fl ** 2)
    return r


def workload(m_list=None):
    return synth.six_regime_sweep(), (m_list or synth.sweep_lengths())


def cells(n, ms):
    prof = sum((n // m) * (n - m + 1) for m in ms)
    ed = sum((n // m) * (m - m // 2 + 1) * (n - m // 2 + 1) for m in ms)
    return prof, ed


def config_dict(n, ms):
    name = ("six-regime sweep, n=100000, m=64..512 step 32, ell=m/2, k=ceil(0.1m), K=4"
            if ms == synth.sweep_lengths() else
            f"six-regime series, n=100000, m in {ms} (a reduced sweep, not the benchmark), ell=m/2, K=4")
    return {"workload": name,
            "n": n, "m_list": ms, "K": K_SNIPPETS, "l2": "flushed (256 MiB write) between timed steps",
            "parallelism": "replicas"}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample(T, ms, block: int, seed: int, cores: int):
    """Oracle (PSF steps, FP64) on a bounded sample: for every m of the sweep,
    ceil(cores * 64 / m) seeded segments over one seeded block of `block`
    positions.  Returns (profile cells, seconds, description)."""
    import oracle
    oracle.set_threads(cores)
    oracle.build()
    rng = np.random.default_rng(seed)
    n = T.shape[0]
    tot_cells, tot_s = 0, 0.0
    for m in ms:
        S, P = n // m, n - m + 1
        nseg = min(S, -(-cores * 64 // m))
        segs = rng.choice(S, nseg, replace=False)
        p_lo = int(rng.integers(0, P - block))
        t0 = time.perf_counter()
        oracle.profiles_range(T, m, m // 2, (m + 9) // 10, segs, p_lo, p_lo + block)
        tot_s += time.perf_counter() - t0
        tot_cells += nseg * block
    desc = (f"every m of the sweep: ceil({cores}*64/m) seeded segments x {block} consecutive positions "
            f"({tot_cells} profile cells), PSF steps in FP64, OpenMP over segments")
    return tot_cells, tot_s, desc


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    s, ms = workload(args.m_list)
    cores = os.cpu_count() or 1
    block = 2048  # the same sample block as the cpu_baseline leg of the GPU arm (about 6 s per step on 16 cores)
    for w in range(args.warmup):
        oracle_sample(s.T, ms, block, 1000 + w, cores)
    times, tot_cells, desc = [], 0, ""
    for st in range(args.steps):
        c, sec, desc = oracle_sample(s.T, ms, block, 2000 + st, cores)
        times.append(sec)
        tot_cells += c
    value = tot_cells / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(s.T.shape[0], ms),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- ranks

def max_over_ranks(seconds: float, dist=None, device="cpu") -> float:
    """The whole job's time: the slowest rank's (every rank calls this after the
    same timed region; replicas only, so this is the one collective)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, cells_per_step: float, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas, each doing `steps` steps of
    `cells_per_step` cells, all done within `seconds` (the slowest rank's time)."""
    return world * cells_per_step * steps / seconds


# ----------------------------------------------------------------------------- serving

def job_ed_cells(job):
    """Algorithmic eq. 9 cells of a serving job: sum over its sweep of S x R x C."""
    return sum((job.n // m) * (m - m // 2 + 1) * (job.n - m // 2 + 1) for m in job.ms)


def job_profile_cells(job):
    return sum((job.n // m) * (job.n - m + 1) for m in job.ms)


def fifo_latencies(arrivals, service):
    """Latencies of one server taking jobs first come, first served."""
    free, out = 0.0, []
    for a, s in zip(arrivals, service):
        start = max(a, free)
        free = start + s
        out.append(free - a)
    return out


def run_serving(args, pastila, device, ed_rate, fp64_ed_rate, age_weight=0.0, policy="share"):
    jobs = synth.serving_jobs(n_jobs=args.serve_jobs, rate=20.0, seed=3)
    series = [j.series() for j in jobs]  # drawn before the clock starts
    ed = np.array([job_ed_cells(j) for j in jobs], dtype=np.float64)
    prof = np.array([job_profile_cells(j) for j in jobs], dtype=np.float64)
    pol = pastila.POLICY_SRPT if policy == "srpt" else pastila.POLICY_SHARE
    # the engine's capacity on this job mix: every job submitted at once, jobs per
    # second of makespan (the mix's lengths reach 768 and its series are short, so
    # it runs below the sweep's cell rate)
    with pastila.Engine(device=device, age_weight_s=age_weight, policy=pol) as e:
        t0 = time.perf_counter()
        ids = [e.submit(T, j.ms, j.K) for T, j in zip(series, jobs)]
        for i in ids:
            e.wait(i)
        closed_s = time.perf_counter() - t0
    capacity = len(jobs) / closed_s
    rate = args.serve_load * capacity  # jobs/s
    arrivals = [j.arrival * 20.0 / rate for j in jobs]
    with pastila.Engine(device=device, age_weight_s=age_weight, policy=pol) as e, ClockSampler(device) as clk:
        t0 = time.perf_counter()
        ids = []
        for T, j, at in zip(series, jobs, arrivals):
            wait = t0 + at - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            ids.append(e.submit(T, j.ms, j.K))
        infos = [e.wait(i) for i in ids]
        st = e.stats()
    assert all(i["state"] == pastila.JOB_DONE for i in infos), "a serving job did not finish"
    lat = np.array([i["t_done"] - i["t_submit"] for i in infos])
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    # latency by job size: thirds of the stream by ED cells
    order = np.argsort(ed, kind="stable")
    by_size = []
    for part in np.array_split(order, 3):
        if part.size == 0:
            continue
        by_size.append({"jobs": int(part.size), "ed_cells_min": float(ed[part].min()),
                        "ed_cells_max": float(ed[part].max()),
                        "latency_p50_s": float(np.percentile(lat[part], 50)),
                        "latency_p99_s": float(np.percentile(lat[part], 99))})
    # the documented stream offers 20 jobs/s; the engine takes `capacity` jobs/s of
    # this mix, so the leg runs the same jobs with the arrival clock scaled to the
    # offered load asked
    out = {"jobs": len(jobs), "arrival_rate_jobs_per_s": rate, "offered_load": args.serve_load,
           "age_weight_s": age_weight, "policy": policy,
           "workload": "serving stream seed 3: n log-uniform [1e4, 5e5], 3-8 planted regimes + N(0, 0.05^2), "
                       "3-10 lengths from {64, 96, ..., 768}, ell = m/2, K in [3, 6]; Poisson arrivals, "
                       "time-scaled from 20 jobs/s to the offered load",
           "documented_rate_jobs_per_s": 20.0, "capacity_jobs_per_s": capacity,
           "capacity_basis": "all jobs submitted at once: jobs / makespan (%.1f s)" % closed_s,
           "sweep_rate_capacity_jobs_per_s": ed_rate / ed.mean(),
           "documented_rate_over_capacity": 20.0 / capacity,
           "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
           "latency_mean_s": float(lat.mean()), "latency_max_s": float(lat.max()),
           "latency_by_job_size": by_size,
           "makespan_s": span, "profile_cells_per_s": float(prof.sum() / span),
           "ed_cells_per_s": float(ed.sum() / span), "waves": st["waves"], "launches": st["launches"],
           "device_busy_frac": st["busy_ms"] / 1e3 / span, "mem_peak_gb": st["mem_peak"] / 1e9,
           "runtime_model": {"waves_observed": st["model_waves"], "wave_rel_err": st["model_rel_err"]},
           "clocks": clk.summary()}
    if fp64_ed_rate:
        lat64 = np.array(fifo_latencies(arrivals, ed / fp64_ed_rate))
        out["fp64_plain_fifo_model"] = {
            "latency_p50_s": float(np.percentile(lat64, 50)), "latency_p99_s": float(np.percentile(lat64, 99)),
            "basis": "same arrivals, one job at a time, service time = job ED cells / the FP64 path's "
                     "measured ED-cell rate on the sweep"}
    return out


def run_serving_plain(args, pastila, device, rate, precision):
    """The serving stream run one job at a time, in arrival order, on handles of
    the given precision (select_length per job, no engine): arrival -> results
    latency measured against the same arrival clock as the engine's run."""
    jobs = synth.serving_jobs(n_jobs=args.serve_jobs, rate=20.0, seed=3)[:args.serve_plain_jobs]
    series = [j.series() for j in jobs]
    arrivals = [j.arrival * 20.0 / rate for j in jobs]
    lat = []
    t0 = time.perf_counter()
    for T, j, at in zip(series, jobs, arrivals):
        wait = t0 + at - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        with pastila.Series(T, device=device, precision=precision) as h:
            h.select_length(j.ms, j.K)
        lat.append(time.perf_counter() - t0 - at)
    lat = np.array(lat)
    return {"precision": "f64" if precision == pastila.FP64 else "f32", "jobs": len(jobs),
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_mean_s": float(lat.mean()), "makespan_s": float(time.perf_counter() - t0),
            "basis": f"measured: the first {len(jobs)} jobs of the serving leg's stream at its arrival times, "
                     "one job at a time in arrival order, select_length on a handle per job"}


def run_multivariate(pastila, device, ms, K, d=3, seeds=(1, 5, 9)):
    """A d-coordinate series (Section 3.1: each coordinate searched on its own,
    Section 3.2), the coordinates six-regime series like the sweep's, through the
    engine in one submission (its coordinates share waves) against the same
    coordinates one after the other through select_length on a handle each.
    Wall time from submission to the last result; both runs once untimed first."""
    T = np.stack([synth.six_regime_sweep(seed=sd).T for sd in seeds[:d]])
    n = T.shape[1]
    prof = d * cells(n, ms)[0]

    def engine_run():
        with pastila.Engine(device=device) as e:
            t0 = time.perf_counter()
            ids = e.submit_multivariate(T, ms, K)
            infos = [e.wait(j) for j in ids]
            res = [e.result(j) for j in ids]
            dt = time.perf_counter() - t0
        assert all(i["state"] == pastila.JOB_DONE for i in infos), "a coordinate did not finish"
        return dt, res, len({i["first_wave"] for i in infos})

    def sequential_run():
        t0 = time.perf_counter()
        res = []
        for c in range(d):
            with pastila.Series(T[c], device=device, precision=pastila.FP32) as h:
                res.append(h.select_length(ms, K))
        return time.perf_counter() - t0, res

    engine_run()
    sequential_run()
    te, re_, first_waves = engine_run()
    ts, rs = sequential_run()
    same = all(a[0] == b[0] and np.array_equal(np.asarray(a[1]), np.asarray(b[1])) and a[2] == b[2]
               for a, b in zip(re_, rs))
    return {"coordinates": d, "n": n, "m_list": ms, "K": K,
            "workload": "d six-regime series (seeds %s), one engine submission" % (list(seeds[:d]),),
            "engine_s": te, "engine_profile_cells_per_s": prof / te, "engine_first_waves": first_waves,
            "sequential_s": ts, "sequential_profile_cells_per_s": prof / ts,
            "results_identical": bool(same),
            "basis": "wall time, submission to last result; sequential = select_length on one handle "
                     "per coordinate, one after the other"}


# ----------------------------------------------------------------------------- GPU arm

def sample_cells(S, P, W, count, rng):
    """Seeded (segment, position) cells of one length: random ones plus the
    first and last segment, the first and last position and both sides of
    every tile boundary (multiples of the tile width W) the sample reaches."""
    segs = list(rng.integers(0, S, count))
    pos = list(rng.integers(0, P, count))
    edges = [0, P - 1] + [q for b in range(W, P, W) for q in (b - 1, b)][:count]
    for i, q in enumerate(edges):
        segs.append([0, S - 1][i % 2] if i < 4 else int(rng.integers(0, S)))
        pos.append(q)
    return np.array(segs, dtype=np.int32), np.array(pos, dtype=np.int64)


def fp32_errors(h, T, ms, res32, res64, dev, count=24, seed=11):
    """Errors of the FP32 results: per length, sampled profile cells (the
    single-length launch with the sweep's tile layout, which computes every cell
    exactly as the batched launch does) against the oracle's pair definition,
    under the tolerance rule; the criterion and m_best against the FP64 GPU path
    (select_length on an FP64 handle), and m_best's snippets."""
    import torch
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    n = T.shape[0]
    per_m, worst = [], 0.0
    Dbuf = torch.empty(max((n // m) * (n - m + 1) for m in ms), dtype=torch.float32, device=dev)
    dmax = torch.zeros(1, dtype=torch.float64, device=dev)
    for m in ms:
        ell, k = m // 2, (m + 9) // 10
        S, P = n // m, n - m + 1
        W = h.tile_layout(m)["W"]
        segs, pos = sample_cells(S, P, W, count, rng)
        h.profiles_device(m, Dbuf.data_ptr(), dmax.data_ptr())
        torch.cuda.synchronize()  # the handle's stream is not torch's
        idx = torch.from_numpy(segs.astype(np.int64) * P + pos).to(dev)
        d32 = Dbuf[idx].double().cpu().numpy()
        dref = oracle.profile_cells(T, m, ell, k, segs, pos)
        r = profile_error_ratio(d32, dref, ell)
        drho = np.abs(d32 ** 2 - dref ** 2) / (2.0 * ell)
        worst = max(worst, float(r.max()) / 1e-4)
        per_m.append({"m": m, "cells": int(r.size), "max_err_over_tol": float(r.max()) / 1e-4,
                      "max_abs_drho": float(drho.max())})
    out = {"tol": 1e-4, "rule": "relative above d_floor = 0.1 sqrt(2 ell), |d^2 - d_ref^2| / (2 d_floor^2) below",
           "profile_cells": {"reference": "oracle pair definition (FP64, CPU)",
                             "sample": f"{count} seeded cells and up to {count} tile-boundary cells per length",
                             "max_err_over_tol": worst, "per_m": per_m}}
    if res64 is not None:
        c32, c64 = np.asarray(res32[1], dtype=np.float64), np.asarray(res64[1], dtype=np.float64)
        rel = np.abs(c32 - c64) / np.maximum(np.abs(c64), 1e-300)
        out["criterion"] = {"reference": "FP64 GPU path", "max_rel_diff": float(rel.max()),
                            "per_m": [float(x) for x in rel]}
        out["m_best"] = {"fp32": int(res32[0]), "fp64": int(res64[0]), "equal": int(res32[0]) == int(res64[0])}
        s32 = [int(r[0]) for r in res32[2]]
        s64 = [int(r[0]) for r in res64[2]]
        out["m_best_snippets"] = {"fp32": s32, "fp64": s64, "equal": s32 == s64}
        # every length's snippets in greedy order (single-length snippets on both handles)
        with pastila_module().Series(T, device=dev.index or 0, precision=pastila_module().FP64) as h64:
            agree = []
            for m in ms:
                a = [int(r[0]) for r in sorted(h.snippets(m, K_SNIPPETS)[0], key=lambda r: r[1])]
                b = [int(r[0]) for r in sorted(h64.snippets(m, K_SNIPPETS)[0], key=lambda r: r[1])]
                agree.append({"m": m, "fp32": a, "fp64": b, "equal": a == b})
        out["snippets_per_m"] = {"reference": "FP64 GPU path, pastila_snippets per length",
                                 "equal_lengths": sum(x["equal"] for x in agree), "lengths": len(agree),
                                 "per_m": agree}
    return out


def pastila_module():
    from paper_2401_13680_b300 import pastila
    return pastila


def run_drift(pastila, device, dev, m=256, K=6, nseg=32, block=512, seed=12):
    """The million-point drift series (8 planted regimes of 50k-250k points plus
    a random walk, m = 256, ell = 128, K = 6): FP32 profiles + greedy snippets
    through the C ABI, timed; the FP64 GPU path timed on the series' first
    125,000 points (1/64 of the ED cells; the full-size FP64 run takes about a
    minute), the FP32 path on the same prefix beside it; FP32 profile cells of
    nseg seeded segments x block consecutive positions against the oracle."""
    import torch
    import oracle
    s = synth.large_drift()
    T = s.T
    n = T.shape[0]
    ell, k = m // 2, (m + 9) // 10
    S, P, R = n // m, n - m + 1, m - ell + 1
    out = {"workload": "drift series, n=1000000, 8 planted regimes + random walk sd 0.01, seed 2; m=256, ell=128, "
                       "k=26, K=6"}
    with pastila.Series(T, device=device, precision=pastila.FP32) as h:
        h.snippets(m, K)  # warm-up: statistics, allocations
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        recs, _, _ = h.snippets(m, K)
        torch.cuda.synchronize()
        t32 = time.perf_counter() - t0
        out["fp32"] = {"seconds": t32, "profile_cells_per_s": S * P / t32,
                       "ed_cells_per_s": S * R * (n - ell + 1) / t32, "snippets": [int(r[0]) for r in recs]}
        rng = np.random.default_rng(seed)
        segs = np.sort(rng.choice(S, nseg, replace=False)).astype(np.int32)
        p_lo = int(rng.integers(0, P - block))
        Dbuf = torch.empty(S * P, dtype=torch.float32, device=dev)
        dmax = torch.zeros(1, dtype=torch.float64, device=dev)
        h.profiles_device(m, Dbuf.data_ptr(), dmax.data_ptr())
        torch.cuda.synchronize()  # the handle's stream is not torch's
        rows = Dbuf.view(S, P)[torch.from_numpy(segs.astype(np.int64)).to(dev), p_lo:p_lo + block]
        d32 = rows.double().cpu().numpy()
        del Dbuf
    oracle.build()
    t0 = time.perf_counter()
    dref = oracle.profiles_range(T, m, ell, k, segs, p_lo, p_lo + block)
    out["oracle_seconds"] = time.perf_counter() - t0
    r = profile_error_ratio(d32, dref, ell)
    out["errors"] = {"cells": int(r.size), "sample": f"{nseg} seeded segments x {block} consecutive positions",
                     "max_err_over_tol": float(r.max()) / 1e-4,
                     "max_abs_drho": float((np.abs(d32 ** 2 - dref ** 2) / (2.0 * ell)).max())}
    # FP32 and FP64 on the first 125,000 points
    Tp = np.ascontiguousarray(T[:125_000])
    np_ = Tp.shape[0]
    ed_p = (np_ // m) * R * (np_ - ell + 1)
    pref = {"n": np_, "ed_cells": ed_p}
    for name, prec in (("fp32", pastila.FP32), ("fp64", pastila.FP64)):
        with pastila.Series(Tp, device=device, precision=prec) as hp:
            hp.profiles(m, want_D=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hp.profiles(m, want_D=False)
            torch.cuda.synchronize()
            pref[name + "_seconds"] = time.perf_counter() - t0
    pref["fp32_over_fp64"] = pref["fp64_seconds"] / pref["fp32_seconds"]
    out["prefix_125k"] = pref
    return out


def run_stress(pastila, device, n, m=128, K=8):
    """The ECG-like stress series (PQRST beats, RR intervals N(800, 40), 12
    morphology regimes, N(0, 0.02^2) noise, seed 4) at n points, one length
    (m = 128, ell = 64, K = 8) through the greedy search without the profile set
    (pastila_snippets_streamed): full passes over the segments, rows recomputed,
    wall time.  At the documented n = 10^7 the profile set of m = 128 would be
    3.1 TB."""
    import torch
    s = synth.ecg_like(n=n)
    T = s.T
    ell = m // 2
    S, R, C = n // m, m - ell + 1, n - ell + 1
    with pastila.Series(T, device=device, precision=pastila.FP32) as h:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        recs, _, _, (passes, rows) = h.snippets_streamed(m, K)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
    pass_ed = S * R * C
    return {"workload": f"ECG-like series, n={n}, 12 regimes, seed 4; m={m}, ell={ell}, k={(m + 9) // 10}, K={K}",
            "seconds": sec, "full_passes": int(passes), "rows_recomputed": int(rows),
            "ed_cells_per_pass": pass_ed,
            "ed_cells_computed": float(pass_ed * passes + rows * R * C),
            "ed_cells_per_s": float(pass_ed * passes + rows * R * C) / sec,
            "snippets": [int(r[0]) for r in recs],
            "documented_n": 10_000_000,
            "projected_pass_seconds_at_documented_n": sec / max(1, passes) * (10_000_000 / n) ** 2}


def run_ours(args):
    import torch
    from paper_2401_13680_b300 import pastila

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    s, ms = workload(args.m_list)
    T = s.T
    n = T.shape[0]
    prof_cells, ed_cells = cells(n, ms)

    # CPU baseline first (rank 0, N = 1 only), before the GPU is busy
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        c, sec, desc = oracle_sample(T, ms, 2048, 7, cores)
        cpu = {"value": c / sec, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": sec}

    stream = torch.cuda.Stream(device=dev)
    T_dev = torch.from_numpy(T).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    torch.cuda.synchronize()
    h = pastila.Series(None, device=local, precision=pastila.FP32, device_ptr=T_dev.data_ptr(), n=n,
                       stream=stream.cuda_stream)

    # autotuner: time candidate tile layouts per length (outside the timed region);
    # the fastest is used by every later call, the serving engine's included
    tune = None
    if not args.no_tune:
        res = h.tune(ms, max_candidates=8)
        tune = {"per_m": [{"m": r["m"], "W": r["W"], "NG": r["NG"], "NT": r["NT"], "GS": r["GS"], "CS": r["CS"], "candidates": r["candidates"],
                           "ms_model": r["ms_model"], "ms_best": r["ms_best"]} for r in res],
                "sample_speedup_over_model": sum(r["ms_model"] for r in res) / sum(r["ms_best"] for r in res),
                "sample": "first min(S, 64) segments of each length, all positions; best of 2 timed launches"}

    def step():
        h.reload_device(T_dev.data_ptr())
        return h.select_length(ms, K_SNIPPETS)

    warm = max(3, args.warmup)
    for _ in range(warm):
        result = step()

    # ---- timed region: device time of each step, L2 flushed in between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    h.set_timing(True)
    l0 = h.kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                starts[i].record(stream)
            result = step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    launches = h.kernel_launches() - l0
    tile_ms, tile_launches, tile_cells_halo = h.tile_time()
    h.set_timing(False)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    tot_s = sum(step_ms) / 1e3
    tot_s = max_over_ranks(tot_s, dist, dev)
    value = replica_rate(world, prof_cells, args.steps, tot_s)
    clocks = clk.summary()

    # ---- end to end through the C ABI: host series in, host results out
    T_host = torch.from_numpy(T).pin_memory().numpy()
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h.reload(T_host)
        h.select_length(ms, K_SNIPPETS)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, dev)
    d2h = 4 + 8 * len(ms) + len(ms) * K_SNIPPETS * 24
    e2e = {"value": replica_rate(world, prof_cells, 1, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s}

    # ---- roofline of the dominant kernel (profile tiles), from its own events:
    # the algorithmic ED cells (S x R x C per length) of all timed launches over
    # their summed device time
    tile_s = tile_ms / 1e3
    achieved = FLOP_PER_ED_CELL * ed_cells * args.steps / tile_s / 1e12
    peak = SM_COUNT_B300 * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    fma32, fma64 = pastila.probe_fma(local)  # measured FMA rates, outside every timed region
    # DRAM bytes of one sweep's tile launches (read + write; the algorithmic bytes are
    # the profile set D, 2.97 GB), from a capture of the current kernel sources only
    traffic, traffic_src = measured_traffic() if ms == synth.sweep_lengths() else (None, "not the full sweep")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per sweep step's tile launches",
                "traffic_source": traffic_src,
                "kernel": "batched_tiles_kernel<float,4> (every length of the sweep; one launch per layout class, "
                          "timed together)",
                "peak_basis": "148 SMs x 128 FP32 lanes x 2 FLOP x 2032 MHz (max SM clock), derived",
                "launches": tile_launches, "avg_launch_ms": tile_ms / max(tile_launches, 1),
                "ed_cells_per_s": ed_cells * args.steps / tile_s,
                "tile_share_of_step": tile_s / tot_s if world == 1 else None,
                "halo_factor": tile_cells_halo / (ed_cells * args.steps),
                "issue_active_ncu": (recorded_capture()[0] or {}).get("issue_active"),
                "fma_measured_tflops": {"fp32": fma32, "fp64": fma64,
                                        "basis": "pastila_probe_fma: 8 independent FMA chains per thread, "
                                                 "8 CTAs of 256 threads per SM, events"},
                "frac_of_measured_fp32_fma": achieved / fma32 if fma32 else None}

    # ---- the plain FP64 one-job GPU path on the same workload (one step)
    fp64 = None
    if not args.no_fp64:
        h64 = pastila.Series(None, device=local, precision=pastila.FP64, device_ptr=T_dev.data_ptr(), n=n,
                             stream=stream.cuda_stream)
        h64.reload_device(T_dev.data_ptr())
        h64.select_length(ms, K_SNIPPETS)  # warm-up: allocations
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(-1.0)
            e0.record(stream)
        h64.reload_device(T_dev.data_ptr())
        r64 = h64.select_length(ms, K_SNIPPETS)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        fp64 = {"value": prof_cells / t64, "unit": UNIT, "ms_per_step": 1e3 * t64, "m_best": r64[0],
                "ed_cells_per_s": ed_cells / t64,
                "speedup_fp32_over_fp64": (prof_cells / (tot_s / args.steps)) / (prof_cells / t64)}
        h64.close()

    # ---- the FP32 path's error, stated per result: profile cells against the oracle,
    # the criterion, m_best and m_best's snippets against the FP64 GPU path
    errors = None
    if not args.no_errors and world == 1:
        errors = fp32_errors(h, T, ms, result, r64 if fp64 else None, dev)

    drift = None
    if not args.no_drift and world == 1:
        drift = run_drift(pastila, local, dev)

    stress = None
    if args.stress and world == 1:
        stress = run_stress(pastila, local, args.stress)

    serving = None
    if args.serve_jobs > 0 and world == 1:
        serving = run_serving(args, pastila, local, ed_cells * args.steps / tot_s,
                              fp64["ed_cells_per_s"] if fp64 else None, args.serve_age_weight,
                              "srpt" if args.serve_policy == "srpt" else "share")
        if args.serve_policy == "both":
            serving["srpt"] = run_serving(args, pastila, local, ed_cells * args.steps / tot_s, None,
                                          args.serve_age_weight, "srpt")
        if args.serve_plain:
            serving["plain_fifo_measured"] = [
                run_serving_plain(args, pastila, local, serving["arrival_rate_jobs_per_s"], prec)
                for prec in (pastila.FP32, pastila.FP64)]

    multi = None
    if not args.no_multi and world == 1:
        multi = run_multivariate(pastila, local, ms, K_SNIPPETS)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(n, ms), "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps, "roofline": roofline,
            "ed_cells_per_s": world * ed_cells * args.steps / tot_s,
            "m_best": result[0], "criterion": [float(x) for x in result[1]],
            "step_ms": step_ms, "fp64_path": fp64, "errors": errors, "drift_series": drift, "stress": stress,
            "serving": serving,
            "multivariate": multi, "autotune": tune}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    h.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the cost model's tile layouts")
    ap.add_argument("--m-list", type=lambda x: [int(v) for v in x.split(",")], default=None,
                    help="comma-separated lengths replacing the sweep (profiling runs on a small case)")
    ap.add_argument("--serve-jobs", type=int, default=32, help="serving-leg jobs (0: no serving leg)")
    ap.add_argument("--serve-age-weight", type=float, default=0.0,
                    help="engine wave shares grow with job age (seconds per unit weight); 0: equal shares")
    ap.add_argument("--serve-policy", choices=["share", "srpt", "both"], default="srpt",
                    help="engine policy of the serving leg: processor sharing, shortest predicted remaining "
                         "first, or both one after the other (same arrivals)")
    ap.add_argument("--serve-plain", action="store_true",
                    help="also run the first --serve-plain-jobs jobs of the serving stream one job at a time on "
                         "FP32 and FP64 handles (slow)")
    ap.add_argument("--serve-plain-jobs", type=int, default=8)
    ap.add_argument("--no-multi", action="store_true", help="skip the multivariate leg")
    ap.add_argument("--no-errors", action="store_true", help="skip the FP32 error block")
    ap.add_argument("--no-drift", action="store_true", help="skip the million-point drift-series leg")
    ap.add_argument("--stress", type=int, default=0,
                    help="points of an ECG-like stress series run through the greedy search without the profile "
                         "set at m = 128, K = 8 (0: skip; the documented size is 10^7)")
    ap.add_argument("--serve-load", type=float, default=0.7,
                    help="offered load of the serving leg, as a fraction of the measured ED-cell rate")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
