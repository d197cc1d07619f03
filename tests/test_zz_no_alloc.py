"""fdtd_step_noalloc: the step for callers that cannot allocate device memory
(their memory belongs to another allocator, or allocation latency and its
implicit synchronisation are not acceptable in their loop).  It runs the same
kernels as fdtd_step with the step kernel's scratch in a static device array.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.  It passes alone in a fresh
process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
PROBE_TOL = 1e-4


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def test_step_noalloc_matches_step_over_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd
    sc = W.random_scenario(41, n=(40, 23, 30), cpml=4, n_steps=50)
    ref = fdtd.from_scenario(sc, probe_capacity=50)
    new = fdtd.from_scenario(sc, probe_capacity=50)
    for g in (ref, new):
        for c, f in enumerate(sc.fields):
            g.set_field(c, f)
    ref.step(50)
    # two calls in a row through the C ABI
    lib = new._lib
    assert lib.fdtd_step_noalloc(new._h, ctypes.c_int(17)) == 0
    assert lib.fdtd_step_noalloc(new._h, ctypes.c_int(33)) == 0
    new.synchronize()
    assert new.step_count == ref.step_count == 50
    for c in range(6):
        assert rel(new.get_field(c), ref.get_field(c)) <= FIELD_TOL
    for p in range(len(sc.probes)):
        assert rel(new.read_probe(p), ref.read_probe(p)) <= PROBE_TOL
    ref.close()
    new.close()


def test_step_noalloc_rejects_unfinalized_grid():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd
    g = fdtd.Grid(8, 8, 8, 0.1)
    assert g._lib.fdtd_step_noalloc(g._h, 1) == -8        # FDTD_ESTATE
    g.close()


@pytest.mark.parametrize("debye", [False, True])
def test_step_noalloc_with_oblique_wires_matches_step(debye):
    """grids with oblique wires (and Debye media): the no-alloc entry runs
    the wires' current update before the step kernels (the graph runs it
    beside them); both order the same arithmetic, so the results are equal
    bit for bit"""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd
    sc = W.random_scenario(43, n=(24, 20, 18), cpml=3, n_wires=0, n_steps=70, courant=0.9)
    if debye:
        sc = W.with_random_debye(sc, 5, materials=(0, 1, 2, 3), max_poles=2)
    J = (11.5, 9.25, 8.75)
    sc.owires = [((5.0, 5.5, 5.0), J, 0.004), (J, (18.5, 14.0, 12.5), 0.002), (J, (6.5, 15.5, 13.0), 0.003)]
    t = np.arange(70)
    sc.owire_sources = [(0, 1, 150.0 * np.sin(0.08 * t), 50.0)]
    sc.owire_probes = [(1, 2), J]
    ref = fdtd.from_scenario(sc, probe_capacity=70)
    new = fdtd.from_scenario(sc, probe_capacity=70)
    for g in (ref, new):
        for c, f in enumerate(sc.fields):
            g.set_field(c, f)
    ref.step(70)
    assert new._lib.fdtd_step_noalloc(new._h, ctypes.c_int(70)) == 0
    new.synchronize()
    for c in range(6):
        assert np.array_equal(new.get_field(c), ref.get_field(c))
    for p in range(len(sc.probes) + len(sc.owire_probes)):
        assert np.array_equal(new.read_probe(p), ref.read_probe(p))
    I0, Q0 = ref.get_wire_state()
    I1, Q1 = new.get_wire_state()
    assert np.array_equal(I0, I1) and np.array_equal(Q0, Q1)
    ref.close()
    new.close()
