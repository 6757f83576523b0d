"""ctypes binding of ``libpastila.so`` (C ABI in ``include/pastila.h``).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  The names follow the C entry points.  There is no CPU fallback:
``load()`` raises if the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ECANCELLED, EBUSY = range(7)
FP32, FP64 = 0, 1
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ECANCELLED", 6: "EBUSY"}


class PastilaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class MParams(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_int32), ("k", ctypes.c_int32)]


class EngineConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("prec", ctypes.c_int), ("mem_budget_bytes", ctypes.c_size_t),
                ("max_active_jobs", ctypes.c_int32), ("wave_ed_cells", ctypes.c_double),
                ("max_waves_in_flight", ctypes.c_int32), ("fail_alloc_at", ctypes.c_int32),
                ("age_weight_s", ctypes.c_double), ("policy", ctypes.c_int32), ("fp32_greedy", ctypes.c_int32),
                ("job_log_path", ctypes.c_char_p)]


POLICY_SHARE, POLICY_SRPT = 0, 1


class JobInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("first_wave", ctypes.c_int64),
                ("last_wave", ctypes.c_int64), ("ed_cells", ctypes.c_double), ("profile_cells", ctypes.c_double),
                ("mem_bytes", ctypes.c_size_t), ("resident_bytes", ctypes.c_size_t),
                ("predicted_ms", ctypes.c_double)]


class EngineCounters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("done", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("waves", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("ed_cells", ctypes.c_double), ("profile_cells", ctypes.c_double), ("busy_ms", ctypes.c_double),
                ("mem_budget", ctypes.c_size_t), ("mem_held", ctypes.c_size_t), ("mem_peak", ctypes.c_size_t),
                ("now", ctypes.c_double), ("model_waves", ctypes.c_uint64), ("model_rel_err", ctypes.c_double)]


class RuntimeModel(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("n_coef", ctypes.c_int32), ("coef", ctypes.c_double * 5),
                ("prior", ctypes.c_double * 5), ("xtx", ctypes.c_double * 25), ("xty", ctypes.c_double * 5),
                ("observations", ctypes.c_uint64), ("err_count", ctypes.c_uint64), ("rel_err", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("W", ctypes.c_int32), ("NG", ctypes.c_int32), ("NT", ctypes.c_int32),
                ("GS", ctypes.c_int32), ("CS", ctypes.c_int32), ("candidates", ctypes.c_int32), ("ms_model", ctypes.c_double), ("ms_best", ctypes.c_double)]


JOB_QUEUED, JOB_ACTIVE, JOB_DONE, JOB_FAILED, JOB_CANCELLED = range(5)


class Snippet(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int32), ("rank", ctypes.c_int32), ("frac", ctypes.c_double),
                ("area_after", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p


def load(path: str | None = None):
    """Build (if stale) and load the library; returns the ctypes handle."""
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(path or _build.build())
        S = ctypes.c_int
        lib.pastila_create.argtypes = [ctypes.POINTER(_vp), _vp, ctypes.c_int64, ctypes.c_int,
                                       ctypes.c_size_t, ctypes.c_int]
        lib.pastila_create.restype = S
        lib.pastila_create_device.argtypes = [ctypes.POINTER(_vp), _vp, ctypes.c_int64, ctypes.c_int,
                                              ctypes.c_size_t, ctypes.c_int, _vp]
        lib.pastila_create_device.restype = S
        lib.pastila_destroy.argtypes = [_vp]
        lib.pastila_destroy.restype = None
        lib.pastila_last_error.argtypes = []
        lib.pastila_last_error.restype = ctypes.c_char_p
        lib.pastila_profiles.argtypes = [_vp, ctypes.c_int32, MParams, _vp, ctypes.POINTER(ctypes.c_double)]
        lib.pastila_profiles.restype = S
        lib.pastila_profiles_device.argtypes = [_vp, ctypes.c_int32, MParams, _vp, _vp]
        lib.pastila_profiles_device.restype = S
        lib.pastila_profiles_batch_device.argtypes = [_vp, _vp, ctypes.c_int32, MParams, _vp, _vp]
        lib.pastila_profiles_batch_device.restype = S
        lib.pastila_stage_status.argtypes = [_vp]
        lib.pastila_stage_status.restype = S
        lib.pastila_set_fp64_ties.argtypes = [_vp, ctypes.c_int]
        lib.pastila_set_fp64_ties.restype = S
        lib.pastila_snippets.argtypes = [_vp, ctypes.c_int32, MParams, ctypes.c_int32,
                                         ctypes.POINTER(Snippet), _vp, _vp]
        lib.pastila_snippets.restype = S
        lib.pastila_select_length.argtypes = [_vp, _vp, ctypes.c_int32, MParams, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32), _vp, ctypes.POINTER(Snippet)]
        lib.pastila_select_length.restype = S
        lib.pastila_reload.argtypes = [_vp, _vp]
        lib.pastila_reload.restype = S
        lib.pastila_reload_device.argtypes = [_vp, _vp]
        lib.pastila_reload_device.restype = S
        lib.pastila_kernel_launches.argtypes = [_vp]
        lib.pastila_kernel_launches.restype = ctypes.c_uint64
        lib.pastila_set_timing.argtypes = [_vp, ctypes.c_int]
        lib.pastila_set_timing.restype = S
        lib.pastila_tile_time.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
        lib.pastila_tile_time.restype = S
        lib.pastila_greedy_noalloc.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _vp, _vp, _vp]
        lib.pastila_greedy_noalloc.restype = S
        lib.pastila_snippets_streamed.argtypes = [_vp, ctypes.c_int32, MParams, ctypes.c_int32,
                                                  ctypes.POINTER(Snippet), _vp, _vp, ctypes.POINTER(ctypes.c_int64)]
        lib.pastila_snippets_streamed.restype = S
        lib.pastila_tune.argtypes = [_vp, _vp, ctypes.c_int32, MParams, ctypes.c_int32, ctypes.POINTER(TuneResult)]
        lib.pastila_tune.restype = S
        lib.pastila_tune_set.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        lib.pastila_tune_set.restype = S
        _i32p = ctypes.POINTER(ctypes.c_int32)
        lib.pastila_tune_get.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                         _i32p, _i32p]
        lib.pastila_tune_get.restype = S
        lib.pastila_plan_layout.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int32, MParams, ctypes.c_size_t,
                                            _vp]
        lib.pastila_plan_layout.restype = S
        lib.pastila_tile_layout.argtypes = [_vp, ctypes.c_int32, MParams, _vp]
        lib.pastila_tile_layout.restype = S
        lib.pastila_tune_clear.argtypes = []
        lib.pastila_tune_clear.restype = None
        lib.pastila_engine_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(EngineConfig)]
        lib.pastila_engine_create.restype = S
        lib.pastila_engine_submit.argtypes = [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int32, MParams,
                                              ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
        lib.pastila_engine_submit.restype = S
        lib.pastila_engine_submit_multi.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int32, _vp, ctypes.c_int32,
                                                    MParams, ctypes.c_int32, _vp]
        lib.pastila_engine_submit_multi.restype = S
        lib.pastila_engine_poll.argtypes = [_vp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(JobInfo)]
        lib.pastila_engine_poll.restype = S
        lib.pastila_engine_result.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), _vp,
                                              ctypes.POINTER(Snippet)]
        lib.pastila_engine_result.restype = S
        lib.pastila_engine_cancel.argtypes = [_vp, ctypes.c_int64]
        lib.pastila_engine_cancel.restype = S
        lib.pastila_engine_release.argtypes = [_vp, ctypes.c_int64]
        lib.pastila_engine_release.restype = S
        lib.pastila_engine_stats.argtypes = [_vp, ctypes.POINTER(EngineCounters)]
        lib.pastila_engine_stats.restype = S
        lib.pastila_engine_destroy.argtypes = [_vp]
        lib.pastila_engine_destroy.restype = None
        lib.pastila_probe_fma.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        lib.pastila_probe_fma.restype = S
        lib.pastila_model_get.argtypes = [ctypes.c_int, ctypes.POINTER(RuntimeModel)]
        lib.pastila_model_get.restype = S
        lib.pastila_model_set.argtypes = [ctypes.POINTER(RuntimeModel)]
        lib.pastila_model_set.restype = S
        lib.pastila_model_observe.argtypes = [ctypes.c_int, _vp, ctypes.c_double]
        lib.pastila_model_observe.restype = S
        lib.pastila_model_reset.argtypes = [ctypes.c_int]
        lib.pastila_model_reset.restype = S
        lib.pastila_model_predict.argtypes = [ctypes.c_int, ctypes.c_int64, _vp, ctypes.c_int32, MParams,
                                              ctypes.c_int32, ctypes.c_size_t, ctypes.c_double,
                                              ctypes.POINTER(ctypes.c_double)]
        lib.pastila_model_predict.restype = S
        _lib = lib
    return _lib


def last_error() -> str:
    return load().pastila_last_error().decode()


def _check(st: int):
    if st != OK:
        raise PastilaError(st, last_error())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def _recs(out):
    return [(s.index, s.rank, s.frac, s.area_after) for s in out]


class Series:
    """A series resident on one GPU (``pastila_create`` / ``pastila_create_device``)."""

    def __init__(self, T, device: int = 0, precision: int = FP32, mem_budget: int = 0,
                 *, device_ptr: int | None = None, n: int | None = None, stream: int | None = None):
        lib = load()
        h = _vp()
        self.precision = precision
        if device_ptr is not None:
            _check(lib.pastila_create_device(ctypes.byref(h), _vp(device_ptr), int(n), device,
                                             mem_budget, precision, _vp(stream or 0)))
            self.n = int(n)
        else:
            T = np.ascontiguousarray(T, dtype=np.float64)
            _check(lib.pastila_create(ctypes.byref(h), _ptr(T), T.shape[0], device, mem_budget, precision))
            self.n = T.shape[0]
        self._h = h

    @property
    def dtype(self):
        return np.float64 if self.precision == FP64 else np.float32

    def close(self):
        if self._h:
            load().pastila_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reload(self, T):
        """``pastila_reload``: new host values, statistics marked stale."""
        T = np.ascontiguousarray(T, dtype=np.float64)
        assert T.shape[0] == self.n
        _check(load().pastila_reload(self._h, _ptr(T)))

    def reload_device(self, ptr: int):
        """``pastila_reload_device``: new values from a device buffer."""
        _check(load().pastila_reload_device(self._h, _vp(ptr)))

    def kernel_launches(self) -> int:
        return int(load().pastila_kernel_launches(self._h))

    def set_timing(self, on: bool):
        _check(load().pastila_set_timing(self._h, 1 if on else 0))

    def tile_time(self):
        """(device ms, launches, ED cells) of the timed tile-kernel launches."""
        ms, n, cells = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        _check(load().pastila_tile_time(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(cells)))
        return ms.value, n.value, cells.value

    def profiles(self, m: int, ell: int = 0, k: int = 0, want_D: bool = True):
        """(D as an S x P array or None, D_max)  -- ``pastila_profiles``."""
        S, P = self.n // m, self.n - m + 1
        D = np.empty((S, P), dtype=self.dtype) if want_D else None
        dmax = ctypes.c_double()
        _check(load().pastila_profiles(self._h, m, MParams(ell, k), _ptr(D) if want_D else None,
                                       ctypes.byref(dmax)))
        return D, dmax.value

    def profiles_device(self, m: int, D_ptr: int, dmax_ptr: int | None = None, ell: int = 0, k: int = 0):
        """Enqueue D into a device buffer (``pastila_profiles_device``)."""
        _check(load().pastila_profiles_device(self._h, m, MParams(ell, k), _vp(D_ptr),
                                              _vp(dmax_ptr) if dmax_ptr else None))

    def profiles_batch_device(self, ms, D_ptrs, dmax_ptr: int | None = None, ell: int = 0, k: int = 0):
        """``pastila_profiles_batch_device``: the profile sets of every m in ms from
        the sweep's batched launch, into the device buffers D_ptrs (one per m)."""
        ms = np.ascontiguousarray(ms, dtype=np.int32)
        ptrs = (ctypes.c_void_p * len(D_ptrs))(*D_ptrs)
        _check(load().pastila_profiles_batch_device(self._h, _ptr(ms), ms.shape[0], MParams(ell, k), ptrs,
                                                    dmax_ptr))

    def set_fp64_ties(self, on: bool):
        """``pastila_set_fp64_ties``: decide near-tied greedy steps of an FP32
        handle on FP64 areas (the default) or on the FP32 areas alone."""
        _check(load().pastila_set_fp64_ties(self._h, 1 if on else 0))

    def stage_status(self):
        """``pastila_stage_status``: raise if a staging wait of enqueued tile work ran
        out (call after synchronising the handle's stream)."""
        _check(load().pastila_stage_status(self._h))

    def snippets(self, m: int, K: int, ell: int = 0, k: int = 0, want_labels: bool = False,
                 want_profiles: bool = False):
        """(records in eq. 8 order, labels or None, chosen profiles or None) --
        ``pastila_snippets``; a record is (index, rank, frac, area_after)."""
        P = self.n - m + 1
        out = (Snippet * K)()
        labels = np.empty(P, dtype=np.int32) if want_labels else None
        prof = np.empty((K, P), dtype=self.dtype) if want_profiles else None
        _check(load().pastila_snippets(self._h, m, MParams(ell, k), K, out,
                                       _ptr(labels) if want_labels else None,
                                       _ptr(prof) if want_profiles else None))
        return _recs(out), labels, prof

    def snippets_streamed(self, m: int, K: int, ell: int = 0, k: int = 0, want_labels: bool = False,
                          want_profiles: bool = False):
        """``pastila_snippets_streamed``: the same results as ``snippets`` without
        the S x P profile set; returns (records, labels, profiles, (passes, rows))."""
        P = self.n - m + 1
        out = (Snippet * K)()
        labels = np.empty(P, dtype=np.int32) if want_labels else None
        prof = np.empty((K, P), dtype=self.dtype) if want_profiles else None
        work = (ctypes.c_int64 * 2)()
        _check(load().pastila_snippets_streamed(self._h, m, MParams(ell, k), K, out,
                                                _ptr(labels) if want_labels else None,
                                                _ptr(prof) if want_profiles else None, work))
        return _recs(out), labels, prof, (work[0], work[1])

    def tune(self, ms, max_candidates: int = 8, ell: int = 0, k: int = 0):
        """``pastila_tune``: time candidate tile layouts per m and keep the fastest
        (process-wide); returns one dict per m."""
        ms = np.ascontiguousarray(ms, dtype=np.int32)
        out = (TuneResult * ms.shape[0])()
        _check(load().pastila_tune(self._h, _ptr(ms), ms.shape[0], MParams(ell, k), max_candidates, out))
        return [{f: getattr(r, f) for f, _ in TuneResult._fields_} for r in out]

    def tile_layout(self, m: int, ell: int = 0, k: int = 0) -> dict:
        """``pastila_tile_layout``: the layout the calls use for length m."""
        out = np.zeros(5, dtype=np.int32)
        _check(load().pastila_tile_layout(self._h, m, MParams(ell, k), _ptr(out)))
        return dict(zip(("W", "NG", "NT", "GS", "CS"), (int(x) for x in out)))

    def select_length(self, ms, K: int, ell: int = 0, k: int = 0):
        """(m_best, crit per m, K records of m_best) -- ``pastila_select_length``."""
        ms = np.ascontiguousarray(ms, dtype=np.int32)
        crit = np.empty(ms.shape[0], dtype=np.float64)
        best = ctypes.c_int32()
        out = (Snippet * K)()
        _check(load().pastila_select_length(self._h, _ptr(ms), ms.shape[0], MParams(ell, k), K,
                                            ctypes.byref(best), _ptr(crit), out))
        return best.value, crit, _recs(out)


class Engine:
    """Serving engine (``pastila_engine_*``): continuous batching of
    select_length jobs on one GPU."""

    def __init__(self, device: int = 0, precision: int = FP32, mem_budget: int = 0, max_active: int = 0,
                 wave_ed_cells: float = 0.0, max_waves_in_flight: int = 0, fail_alloc_at: int = 0,
                 age_weight_s: float = 0.0, policy: int = POLICY_SHARE, fp32_greedy: bool = False,
                 job_log: str | None = None):
        lib = load()
        cfg = EngineConfig(device, precision, mem_budget, max_active, wave_ed_cells, max_waves_in_flight,
                           fail_alloc_at, age_weight_s, policy, 1 if fp32_greedy else 0,
                           job_log.encode() if job_log else None)
        h = _vp()
        _check(lib.pastila_engine_create(ctypes.byref(h), ctypes.byref(cfg)))
        self._h = h
        self._sizes = {}

    def close(self):
        if self._h:
            load().pastila_engine_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, T, ms, K: int, ell: int = 0, k: int = 0) -> int:
        """Queues a job; returns its id."""
        T = np.ascontiguousarray(T, dtype=np.float64)
        ms = np.ascontiguousarray(ms, dtype=np.int32)
        job = ctypes.c_int64()
        _check(load().pastila_engine_submit(self._h, _ptr(T), T.shape[0], _ptr(ms), ms.shape[0], MParams(ell, k),
                                            K, ctypes.byref(job)))
        self._sizes[job.value] = (ms.shape[0], K)
        return job.value

    def submit_multivariate(self, T, ms, K: int, ell: int = 0, k: int = 0) -> list:
        """Queues one job per coordinate of a (d, n) series in one step
        (``pastila_engine_submit_multi``); returns the d job ids."""
        T = np.ascontiguousarray(np.atleast_2d(T), dtype=np.float64)
        ms = np.ascontiguousarray(ms, dtype=np.int32)
        d, n = T.shape
        ids = np.zeros(d, dtype=np.int64)
        _check(load().pastila_engine_submit_multi(self._h, _ptr(T), n, d, _ptr(ms), ms.shape[0], MParams(ell, k),
                                                  K, _ptr(ids)))
        for j in ids:
            self._sizes[int(j)] = (ms.shape[0], K)
        return [int(j) for j in ids]

    def poll(self, job: int, timeout_ms: int = 0):
        """(final?, JobInfo as a dict)."""
        info = JobInfo()
        st = load().pastila_engine_poll(self._h, job, timeout_ms, ctypes.byref(info))
        if st not in (OK, ETIMEOUT):
            _check(st)
        return st == OK, {f: getattr(info, f) for f, _ in JobInfo._fields_}

    def wait(self, job: int):
        return self.poll(job, -1)[1]

    def result(self, job: int):
        """(m_best, crit per m, K records of m_best) of a finished job."""
        n_m, K = self._sizes.get(job, (64, 64))  # an unknown job is the library's error to report
        crit = np.empty(n_m, dtype=np.float64)
        out = (Snippet * K)()
        best = ctypes.c_int32()
        _check(load().pastila_engine_result(self._h, job, ctypes.byref(best), _ptr(crit), out))
        return best.value, crit, _recs(out)

    def cancel(self, job: int):
        _check(load().pastila_engine_cancel(self._h, job))

    def release(self, job: int):
        _check(load().pastila_engine_release(self._h, job))
        self._sizes.pop(job, None)

    def stats(self) -> dict:
        c = EngineCounters()
        _check(load().pastila_engine_stats(self._h, ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in EngineCounters._fields_}


def plan_layout(precision: int, n: int, m: int, smem_limit: int, ell: int = 0, k: int = 0) -> dict:
    """``pastila_plan_layout``: the layout chosen for a length, without a device."""
    out = np.zeros(8, dtype=np.int32)
    _check(load().pastila_plan_layout(precision, n, m, MParams(ell, k), smem_limit, _ptr(out)))
    return dict(zip(("W", "NG", "NT", "GS", "CS", "Rg", "Rh", "bytes"), (int(x) for x in out)))


def probe_fma(device: int = 0) -> tuple:
    """``pastila_probe_fma``: measured (FP32, FP64) FMA rates in TFLOP/s."""
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    _check(load().pastila_probe_fma(device, ctypes.byref(f32), ctypes.byref(f64)))
    return f32.value, f64.value


def model_get(precision: int) -> dict:
    """``pastila_model_get``: the runtime model of a precision, as a dict of
    numpy arrays (coef, prior, xtx 5x5, xty) and counts."""
    r = RuntimeModel()
    _check(load().pastila_model_get(precision, ctypes.byref(r)))
    return {"prec": r.prec, "coef": np.array(r.coef[:]), "prior": np.array(r.prior[:]),
            "xtx": np.array(r.xtx[:]).reshape(5, 5), "xty": np.array(r.xty[:]),
            "observations": int(r.observations), "err_count": int(r.err_count), "rel_err": r.rel_err}


def model_set(model: dict):
    """``pastila_model_set``: warm start from a dict as model_get returns it."""
    r = RuntimeModel()
    r.prec = int(model["prec"])
    r.n_coef = int(model.get("n_coef", 5))
    r.prior[:] = [float(x) for x in np.asarray(model["prior"], dtype=np.float64).ravel()]
    r.xtx[:] = [float(x) for x in np.asarray(model["xtx"], dtype=np.float64).ravel()]
    r.xty[:] = [float(x) for x in np.asarray(model["xty"], dtype=np.float64).ravel()]
    r.observations = int(model.get("observations", 0))
    _check(load().pastila_model_set(ctypes.byref(r)))


def model_observe(precision: int, features, ms: float):
    """``pastila_model_observe``: one measured unit of work (5 features, ms)."""
    f = np.ascontiguousarray(features, dtype=np.float64)
    if f.shape != (5,):
        raise ValueError("features must have 5 entries")
    _check(load().pastila_model_observe(precision, _ptr(f), ms))


def model_reset(precision: int):
    """``pastila_model_reset``: forget every observation of a precision."""
    _check(load().pastila_model_reset(precision))


def model_predict(precision: int, n: int, ms, K: int, smem_limit: int, ell: int = 0, k: int = 0,
                  wave_ed_cells: float = 0.0) -> float:
    """``pastila_model_predict``: predicted device time (ms) of a job, without a device."""
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    out = ctypes.c_double()
    _check(load().pastila_model_predict(precision, n, _ptr(ms), ms.shape[0], MParams(ell, k), K, smem_limit,
                                        wave_ed_cells, ctypes.byref(out)))
    return out.value


def tune_set(precision: int, m: int, ell: int, k: int, W: int, NG: int, GS: int, CS: int = 1):
    """``pastila_tune_set``: one entry of the tuned layout table."""
    _check(load().pastila_tune_set(precision, m, ell, k, W, NG, GS, CS))


def tune_get(precision: int, m: int, ell: int, k: int):
    """``pastila_tune_get``: (W, NG, GS, CS) of an entry of the tuned layout table."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(load().pastila_tune_get(precision, m, ell, k, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def tune_clear():
    """``pastila_tune_clear``: back to the cost model's layouts."""
    load().pastila_tune_clear()


def greedy_noalloc(D_ptr: int, S: int, P: int, K: int, chosen_ptr: int, area_ptr: int,
                   stream: int | None = None):
    """``pastila_greedy_noalloc``: greedy search on a device profile set, with
    the library's fixed scratch; enqueued on ``stream``, not waited for."""
    _check(load().pastila_greedy_noalloc(_vp(D_ptr), S, P, K, _vp(chosen_ptr), _vp(area_ptr),
                                         _vp(stream or 0)))


def exported_symbols():
    """Names of the entry points declared in include/pastila.h."""
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pastila.h")
    return sorted(set(re.findall(r"\b(pastila_[a-z_]+)\s*\(", open(hdr).read())))
