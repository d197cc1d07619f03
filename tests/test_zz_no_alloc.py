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
    # the same kernels on the same inputs: equal bit for bit (the graph runs
    # the z-layer launch beside the interior one, this entry point after it;
    # they write disjoint planes)
    for c in range(6):
        assert np.array_equal(new.get_field(c), ref.get_field(c))
    for p in range(len(sc.probes)):
        assert np.array_equal(new.read_probe(p), ref.read_probe(p))
    ref.close()
    new.close()


def test_step_noalloc_alternating_grids_on_two_streams():
    """a grid with a CPML (two step launches, four counters) and one without
    (one launch, two counters) stepped in turn through the shared static
    scratch, each on its own stream: the error flag has a slot of its own, so
    synchronising one grid while the other's steps run reads no live counter
    and reports nothing, and both grids end equal to fdtd_step bit for bit"""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd
    sa = W.random_scenario(44, n=(40, 23, 30), cpml=4, n_steps=90)
    sb = W.random_scenario(45, n=(33, 20, 17), n_steps=90)
    st_a, st_b = torch.cuda.Stream(), torch.cuda.Stream()
    refs, news = [], []
    for sc, st in ((sa, st_a), (sb, st_b)):
        r = fdtd.from_scenario(sc, probe_capacity=90)
        n = fdtd.from_scenario(sc, stream=st, probe_capacity=90)
        for g in (r, n):
            for c, f in enumerate(sc.fields):
                g.set_field(c, f)
        r.step(90)
        refs.append(r)
        news.append(n)
    a, b = news
    lib = a._lib
    for na, nb in ((30, 20), (25, 40), (35, 30)):
        assert lib.fdtd_step_noalloc(b._h, ctypes.c_int(nb)) == 0
        assert lib.fdtd_synchronize(b._h) == 0
        # a's steps are queued on its own stream while b synchronises
        assert lib.fdtd_step_noalloc(a._h, ctypes.c_int(na)) == 0
        assert lib.fdtd_synchronize(b._h) == 0
        assert lib.fdtd_synchronize(a._h) == 0
    for sc, r, n in zip((sa, sb), refs, news):
        assert n.step_count == r.step_count == 90
        for c in range(6):
            assert np.array_equal(n.get_field(c), r.get_field(c))
        for p in range(len(sc.probes)):
            assert np.array_equal(n.read_probe(p), r.read_probe(p))
        r.close()
        n.close()


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
