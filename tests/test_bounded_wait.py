"""The tile kernels' one wait (for the bulk copies that stage a tile) is
bounded: when it runs out, the tile stores a host-visible flag, still reaches
every barrier, and the call that synchronises reports ETIMEOUT; the context
stays usable.  The test makes the wait run out on purpose the allowed way: with
PASTILA_TEST_STAGE_WAIT=timeout at creation, every tile also waits on a barrier
phase that nothing completes, with a limit of about half a millisecond.  No
fault, trap or endless loop is involved."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_handle_reports_a_wait_that_ran_out(lib, monkeypatch):
    from paper_2401_13680_b300 import pastila
    T = synth.white_noise(3, 2000)
    monkeypatch.setenv("PASTILA_TEST_STAGE_WAIT", "timeout")
    with pastila.Series(T, precision=pastila.FP32) as h:
        with pytest.raises(pastila.PastilaError, match="ETIMEOUT"):
            h.profiles(64)
        with pytest.raises(pastila.PastilaError, match="ETIMEOUT"):
            h.select_length([64, 96], 2)
    monkeypatch.delenv("PASTILA_TEST_STAGE_WAIT")
    # the same device and process go on: a new handle computes normally
    with pastila.Series(T, precision=pastila.FP32) as h:
        D, dmax = h.profiles(64)
        assert np.isfinite(D).all() and 0 < dmax <= 2 * np.sqrt(32) + 1e-4
        with pastila.Series(T, precision=pastila.FP64) as h64:
            D64, _ = h64.profiles(64)
        assert np.max(np.abs(D - D64)) < 1e-2


def test_engine_fails_its_jobs_with_etimeout_and_a_new_engine_serves(lib, monkeypatch):
    from paper_2401_13680_b300 import pastila
    T = synth.white_noise(4, 3000)
    monkeypatch.setenv("PASTILA_TEST_STAGE_WAIT", "timeout")
    with pastila.Engine() as e:
        j = e.submit(T, [64, 128], 2)
        info = e.wait(j)
        assert info["state"] == pastila.JOB_FAILED and info["status"] == pastila.ETIMEOUT
        with pytest.raises(pastila.PastilaError, match="ETIMEOUT"):
            e.result(j)
    monkeypatch.delenv("PASTILA_TEST_STAGE_WAIT")
    with pastila.Engine() as e:
        j = e.submit(T, [64, 128], 2)
        assert e.wait(j)["state"] == pastila.JOB_DONE
        with pastila.Series(T, precision=pastila.FP32) as h:
            ref = h.select_length([64, 128], 2)
        got = e.result(j)
        assert got[0] == ref[0]
        np.testing.assert_array_equal(got[1], ref[1])
