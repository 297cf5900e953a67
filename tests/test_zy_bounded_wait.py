"""Failure detection of bounded device waits, exercised on the GPU without a fault.

Every wait of the library's kernels on another agent is bounded by the GPU's
global timer and reports PF_ETIMEOUT when it runs out.  pf_probe_bounded_wait
runs that bounded wait (20 ms limit) on a barrier of its own with no other
work in flight: completed first, the wait returns PF_OK at once; left
incomplete, only its limit can end it, and the call returns PF_ETIMEOUT with
the device still usable -- the next filter step gives the same results as on
a device that never saw a timeout.  The file is collected late so that a
failure here leaves the other tests run.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1407_8071_gb300 import pf, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _filter_run(y32):
    with pf.EnsembleFilter(W.lorenz63(), 3, 256, 5) as f:
        for t in range(len(y32)):
            f.step(y32[t])
        return f.get_state(), f.estimate(pf.PF_STAT_MEAN, var=1)


def test_a_bounded_wait_that_runs_out_reports_a_timeout_and_leaves_the_device_usable():
    _, y = oracle.simulate(W.lorenz63(), 3, W.SEED_LORENZ_OBS)
    y32 = y.astype(np.float32)
    x0, e0 = _filter_run(y32)
    assert pf.pf_probe_bounded_wait(True) == pf.PF_OK
    for stream in (None, torch.cuda.Stream().cuda_stream):
        t0 = time.perf_counter()
        assert pf.pf_probe_bounded_wait(False, stream) == pf.PF_ETIMEOUT
        dt = time.perf_counter() - t0
        assert 0.015 <= dt < 5.0, dt  # the 20 ms limit, not a hang
        assert b"20 ms" in (pf.lib().pf_last_error(None) or b"")
    assert pf.pf_probe_bounded_wait(True) == pf.PF_OK
    x1, e1 = _filter_run(y32)
    assert np.array_equal(x0, x1) and np.array_equal(e0, e1)
