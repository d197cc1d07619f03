"""Failure detection on the GPU without a fault: a bounded wait that nothing
completes gives up, the host reads the timeout status, and the context keeps
working (the step kernel's waits use the same routine)."""
import ctypes
import time

import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd as F
    return F


def test_bounded_wait_times_out_and_context_survives(fdtd):
    import torch
    from paper_2207_06908_gb300 import _lib
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    rc = lib.fdtd_selftest_wait(0.02, stream)
    dt = time.perf_counter() - t0
    assert rc == -6                         # FDTD_ETIMEOUT
    assert 0.02 <= dt < 2.0
    assert lib.fdtd_selftest_wait(0.0, stream) == -1
    # the context still runs the solver correctly
    sc = W.random_scenario(3, n=(20, 13, 18), cpml=3, n_steps=12)
    g = fdtd.from_scenario(sc, probe_capacity=12)
    for c, f in enumerate(sc.fields):
        g.set_field(c, f)
    g.step(12)
    g.synchronize()
    assert all(np.isfinite(g.get_field(c)).all() for c in range(6))
    g.close()


def test_watchdog_reports_divergence_within_its_period(fdtd):
    """a NaN written into one field from the host (no fault: an ordinary
    upload) is found by the watchdog's next check; the synchronising call
    returns FDTD_EDIVERGED once, within one period, and a clean grid beside
    it with the same period reports nothing"""
    from paper_2207_06908_gb300._lib import FdtdError
    sc = W.random_scenario(5, n=(24, 17, 20), cpml=3, n_steps=128)
    bad = fdtd.from_scenario(sc, probe_capacity=128)
    good = fdtd.from_scenario(sc, probe_capacity=128)
    for g in (bad, good):
        g.set_watchdog(32)
        for c, f in enumerate(sc.fields):
            g.set_field(c, f)
    # 40 clean steps: one check at step 32, nothing to report
    bad.step(40)
    bad.synchronize()
    ez = bad.get_field(2)
    ez[10, 8, 12] = np.nan
    bad.set_field(2, ez)
    # steps 40 .. 63: the next check (step 64) has not run yet
    bad.step(23)
    bad.synchronize()
    bad.step(1)                             # reaches 64: the check runs after this step
    with pytest.raises(FdtdError) as ei:
        bad.synchronize()
    assert ei.value.code == -7              # FDTD_EDIVERGED
    bad.synchronize()                       # reported once per detection
    good.step(128)
    good.synchronize()
    assert all(np.isfinite(good.get_field(c)).all() for c in range(6))
    # off: no report
    bad.set_watchdog(0)
    bad.step(64)
    bad.synchronize()
    bad.close()
    good.close()
