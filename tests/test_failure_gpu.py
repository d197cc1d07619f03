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
