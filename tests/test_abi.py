"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/pastila.h.  CPU only: no call here reaches a kernel."""
import ctypes
import subprocess

import numpy as np

from paper_2401_13680_b300 import build, pastila


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    declared = pastila.exported_symbols()
    assert len(declared) >= 13
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    lib = pastila.load()
    for s in declared:
        assert getattr(lib, s) is not None


def test_host_side_argument_validation():
    lib = pastila.load()
    h = ctypes.c_void_p()
    # NULL series is rejected before any device call
    assert lib.pastila_create(ctypes.byref(h), None, 100, 0, 0, pastila.FP32) == pastila.EINVAL
    assert "T is NULL" in pastila.last_error()
    T = np.array([0.0, 1.0, np.nan, 3.0, 4.0])
    assert lib.pastila_create(ctypes.byref(h), T.ctypes.data_as(ctypes.c_void_p), 5, 0, 0,
                              pastila.FP32) == pastila.EINVAL
    assert "not finite" in pastila.last_error()
    assert lib.pastila_create(None, T.ctypes.data_as(ctypes.c_void_p), 5, 0, 0, pastila.FP32) \
        == pastila.EINVAL
    # a NULL handle is an argument error on every entry point
    assert lib.pastila_profiles(None, 64, pastila.MParams(0, 0), None, None) == pastila.EINVAL
    assert lib.pastila_stage_status(None) == pastila.EINVAL
    assert lib.pastila_profiles_batch_device(None, None, 0, pastila.MParams(0, 0), None, None) == pastila.EINVAL
    assert lib.pastila_snippets(None, 64, pastila.MParams(0, 0), 2, None, None, None) == pastila.EINVAL
    assert lib.pastila_select_length(None, None, 0, pastila.MParams(0, 0), 2, None, None, None) \
        == pastila.EINVAL
    assert lib.pastila_reload(None, None) == pastila.EINVAL
    assert lib.pastila_set_timing(None, 1) == pastila.EINVAL
    assert lib.pastila_kernel_launches(None) == 0
    lib.pastila_destroy(None)  # no-op


def test_engine_host_side_validation():
    lib = pastila.load()
    e = ctypes.c_void_p()
    assert lib.pastila_engine_create(None, None) == pastila.EINVAL
    bad = pastila.EngineConfig(0, 7, 0, 0, 0.0, 0, 0, 0.0)
    assert lib.pastila_engine_create(ctypes.byref(e), ctypes.byref(bad)) == pastila.EINVAL
    assert "precision" in pastila.last_error()
    bad = pastila.EngineConfig(0, pastila.FP32, 0, 1000, 0.0, 0, 0, 0.0)
    assert lib.pastila_engine_create(ctypes.byref(e), ctypes.byref(bad)) == pastila.EINVAL
    bad = pastila.EngineConfig(0, pastila.FP32, 0, 0, 0.0, 0, 0, 0.0, 5)
    assert lib.pastila_engine_create(ctypes.byref(e), ctypes.byref(bad)) == pastila.EINVAL
    assert "policy" in pastila.last_error()
    job = ctypes.c_int64()
    T = np.zeros(100)
    ms = np.array([16], dtype=np.int32)
    assert lib.pastila_engine_submit(None, T.ctypes.data_as(ctypes.c_void_p), 100,
                                     ms.ctypes.data_as(ctypes.c_void_p), 1, pastila.MParams(0, 0), 2,
                                     ctypes.byref(job)) == pastila.EINVAL
    ids = np.zeros(2, dtype=np.int64)
    assert lib.pastila_engine_submit_multi(None, T.ctypes.data_as(ctypes.c_void_p), 50, 2,
                                           ms.ctypes.data_as(ctypes.c_void_p), 1, pastila.MParams(0, 0), 2,
                                           ids.ctypes.data_as(ctypes.c_void_p)) == pastila.EINVAL
    assert lib.pastila_engine_poll(None, 1, 0, None) == pastila.EINVAL
    assert lib.pastila_engine_result(None, 1, None, None, None) == pastila.EINVAL
    assert lib.pastila_engine_cancel(None, 1) == pastila.EINVAL
    assert lib.pastila_engine_release(None, 1) == pastila.EINVAL
    assert lib.pastila_engine_stats(None, None) == pastila.EINVAL
    lib.pastila_engine_destroy(None)  # no-op


def test_no_device_means_an_error_not_a_fallback():
    """There is no CPU path: where no GPU is visible, every entry point that
    needs one reports ECUDA instead of computing anything."""
    import pytest
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    T = np.random.default_rng(0).normal(size=1000)
    for make in (lambda: pastila.Series(T), lambda: pastila.Series(T, precision=pastila.FP64),
                 lambda: pastila.Engine(), lambda: pastila.probe_fma(0)):
        with pytest.raises(pastila.PastilaError, match="ECUDA"):
            make()
