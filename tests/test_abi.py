"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/fdtd.h declares (CPU; no compute calls)."""
import ctypes
import os
import re

from paper_2207_06908_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fdtd_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_oracle_builds():
    from oracle import oracle
    assert os.path.exists(oracle.build())


def _lib():
    from paper_2207_06908_gb300 import _lib as L
    _build.build()
    return L.load()


def _grid(lib, n=(8, 8, 8), dx=0.1, S=0.99, cpml=None):
    h = ctypes.c_void_p()
    rc = lib.fdtd_create_grid(n[0], n[1], n[2], dx, S, cpml, None, ctypes.byref(h))
    return rc, h


def test_host_argument_checks():
    """Host-side validation of the C ABI (no CUDA call is made)."""
    lib = _lib()
    rc, h = _grid(lib, S=1.01)
    assert rc == -2 and not h.value                      # FDTD_ECOURANT
    rc, h = _grid(lib, n=(1, 8, 8))
    assert rc == -1
    rc, h = _grid(lib)
    assert rc == 0
    try:
        wid = ctypes.c_int()
        assert lib.fdtd_add_wire(h, 2, 2, 1, 2, 2, 6, 0.005, ctypes.byref(wid)) == 0
        assert lib.fdtd_add_wire(h, 2, 2, 1, 3, 2, 6, 0.005, None) == -1          # not axis-aligned
        assert lib.fdtd_add_wire(h, 0, 2, 1, 0, 2, 6, 0.005, None) == -1          # on a wall
        assert lib.fdtd_add_wire(h, 2, 2, 1, 2, 2, 6, 0.024, None) == -1          # thicker than 0.23 dx
        assert b"0.23" in lib.fdtd_last_error(h)
        cur = (ctypes.c_double * 4)(1, 2, 3, 4)
        assert lib.fdtd_add_source(h, 3, 3, 3, 2, 0.0, cur, 4, None) == 0
        assert lib.fdtd_add_source(h, 3, 3, 3, 2, 50.0, cur, 4, None) == 0         # non-ideal (parallel R)
        assert lib.fdtd_add_source(h, 3, 3, 3, 2, -1.0, cur, 4, None) == -1        # negative resistance
        assert lib.fdtd_add_voltage_source(h, 3, 3, 3, 2, 0.0, cur, 4, None) == 0  # ideal voltage source
        assert lib.fdtd_add_lumped(h, 3, 3, 4, 2, 50.0, 0.0, None) == 0
        assert lib.fdtd_add_lumped(h, 3, 3, 4, 2, 0.0, 0.0, None) == -1            # no element
        assert lib.fdtd_add_lumped(h, 0, 3, 4, 2, 50.0, 0.0, None) == -1           # wall edge
        assert lib.fdtd_add_source(h, 0, 3, 3, 2, 0.0, cur, 4, None) == -1         # wall edge
        assert lib.fdtd_add_probe(h, 0, 3, 3, 3, 2, 5, None) == 0
        assert lib.fdtd_add_probe(h, 0, 3, 3, 3, 2, 6, None) == -1                 # path leaves grid
        assert lib.fdtd_add_probe(h, 1, 0, 3, 3, 2, 1, None) == -1                 # loop needs i >= 1
        ns = ctypes.c_int()
        assert lib.fdtd_add_wire_path(h, 2, 2, 2, 5, 4, 6, 0.004, ctypes.byref(ns)) == 0 and ns.value >= 3
        assert lib.fdtd_add_wire_path(h, 2, 2, 2, 2, 2, 2, 0.004, None) == -1       # zero length
        assert lib.fdtd_add_wire_path(h, 2, 2, 2, 0, 5, 6, 0.004, None) == -1       # reaches a wall
        assert lib.fdtd_step(h, 1) == -8                                           # not finalized
        nbytes = ctypes.c_size_t()
        assert lib.fdtd_save_state(h, None, ctypes.byref(nbytes)) == -8            # not finalized
        assert lib.fdtd_load_state(h, b"x" * 64, 64) == -8
        assert lib.fdtd_save_state(None, None, ctypes.byref(nbytes)) == -1
        nb = ctypes.c_size_t()
        assert lib.fdtd_arena_bytes(h, 100, ctypes.byref(nb)) == 0 and nb.value > 12 * 8 * 8 * 8 * 4
    finally:
        lib.fdtd_destroy(h)


def test_too_many_classes_rejected_before_any_device_work():
    """More than 256 distinct coefficient sets -> FDTD_ECLASSES (host-side
    class building runs before any allocation)."""
    import numpy as np
    from paper_2207_06908_gb300._lib import Material
    lib = _lib()
    rc, h = _grid(lib, n=(24, 24, 24))
    try:
        rng = np.random.default_rng(0)
        cm = rng.integers(0, 40, size=24 ** 3).astype(np.uint8)
        mats = (Material * 40)(*[Material(1.0 + q, 0.001 * q, 1.0) for q in range(40)])
        assert lib.fdtd_set_materials(h, cm.ctypes.data_as(ctypes.c_void_p), mats, 40) == 0
        assert lib.fdtd_finalize(h, 0, None, 0) == -5
        assert lib.fdtd_set_materials(h, cm.ctypes.data_as(ctypes.c_void_p), mats, 30) == -1
    finally:
        lib.fdtd_destroy(h)


def test_oblique_wire_host_checks():
    """Oblique wires (host only): argument checks, segment counts
    (round(length in cells)), junctions join coinciding end points, the
    segment and probe ids, and errors for bad segments."""
    from paper_2207_06908_gb300 import _lib as L
    lib = L.load()
    h = ctypes.c_void_p()
    assert lib.fdtd_create_grid(20, 18, 16, 0.1, 0.99, None, None, ctypes.byref(h)) == 0
    try:
        wid, ns, nn = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ok = lib.fdtd_add_oblique_wire
        assert ok(h, 3.0, 4.0, 5.0, 3.0, 4.0, 5.2, 0.002, None) == -1          # shorter than half a cell
        assert ok(h, 3.0, 4.0, 5.0, 21.0, 4.0, 5.0, 0.002, None) == -1         # leaves the grid
        assert ok(h, 3.0, 4.0, 5.0, 9.0, 4.0, 5.0, 0.011, None) == -1          # radius above 0.1 dx
        assert ok(h, 3.3, 4.1, 3.7, 11.2, 9.6, 8.4, 0.002, ctypes.byref(wid)) == 0 and wid.value == 0
        assert lib.fdtd_wire_counts(h, ctypes.byref(ns), ctypes.byref(nn)) == 0
        length = ((11.2 - 3.3) ** 2 + (9.6 - 4.1) ** 2 + (8.4 - 3.7) ** 2) ** 0.5
        assert ns.value == round(length) and nn.value == ns.value + 1
        assert ok(h, 11.2, 9.6, 8.4, 12.5, 3.2, 5.0, 0.003, ctypes.byref(wid)) == 0 and wid.value == 1
        lib.fdtd_wire_counts(h, ctypes.byref(ns), ctypes.byref(nn))
        assert nn.value == ns.value + 1                                        # one tree: the end point joined
        assert ok(h, 5.0, 5.0, 0.0, 5.0, 5.0, 4.0, 0.004, None) == 0           # grounded on z = 0
        v = (ctypes.c_double * 4)(1.0, 2.0, 3.0, 4.0)
        sid, pid = ctypes.c_int(), ctypes.c_int()
        assert lib.fdtd_add_wire_voltage_source(h, 1, 0, 0.0, v, 4, ctypes.byref(sid)) == 0 and sid.value == 0
        assert lib.fdtd_add_wire_voltage_source(h, 1, 0, 400.0, v, 4, ctypes.byref(sid)) == 0 and sid.value == 1
        assert lib.fdtd_add_wire_voltage_source(h, 1, 0, -1.0, v, 4, None) == -1
        assert lib.fdtd_add_wire_voltage_source(h, 1, 99, 0.0, v, 4, None) == -1
        assert lib.fdtd_add_wire_voltage_source(h, 7, 0, 0.0, v, 4, None) == -1
        assert lib.fdtd_add_probe(h, 0, 2, 2, 2, 2, 1, ctypes.byref(pid)) == 0 and pid.value == 0
        assert lib.fdtd_add_wire_probe(h, 0, 3, ctypes.byref(pid)) == 0 and pid.value == 1
        assert lib.fdtd_add_wire_probe(h, 2, 4, None) == -1                    # the grounded wire has 4
    finally:
        lib.fdtd_destroy(h)


def test_thick_oblique_wire_needs_a_smaller_courant_number():
    """a wire along a node line with ln(R/a) = 1 caps the Courant number
    below 0.99: finalize refuses before any device work and names the cap"""
    import math
    from paper_2207_06908_gb300 import _lib as L
    lib = L.load()
    a = 0.1 * math.exp(-0.57721566490153286) / (2 * math.sqrt(2)) / math.e
    for courant, rc in ((0.99, -2), (0.85, None)):
        h = ctypes.c_void_p()
        assert lib.fdtd_create_grid(14, 14, 14, 0.1, courant, None, None, ctypes.byref(h)) == 0
        try:
            assert lib.fdtd_add_oblique_wire(h, 1.0, 7.0, 7.0, 13.0, 7.0, 7.0, a, None) == 0
            lim = ctypes.c_double()
            assert lib.fdtd_wire_courant_limit(h, ctypes.byref(lim)) == 0
            assert abs(lim.value - 1 / math.sqrt(1 + 2 * math.exp(-1.89))) < 1e-9
            if rc is not None:
                assert lib.fdtd_finalize(h, 0, None, 0) == rc
                assert b"courant" in lib.fdtd_last_error(h)
        finally:
            lib.fdtd_destroy(h)


def test_inclined_grounding_domains_fit_and_stay_below_the_wire_limit():
    """every domain of the inclined-rod batched workload: the riser and leads
    are accepted, the inclined rod lies inside the domain and joins the
    riser's bottom node, and the Courant number the workload runs at is
    below the domain's oblique-wire limit (so finalize accepts it)"""
    from paper_2207_06908_gb300 import workloads as W
    lib = _lib()
    scs = W.config4_inclined(n_steps=10)
    assert len(scs) == 256
    for sc in scs:
        (p0, p1, r), = sc.owires
        riser = sc.wires[0]
        assert riser[0] == tuple(int(v) for v in p0) and riser[0][:2] == riser[1][:2]   # rod top = riser bottom
        assert all(sc.cpml + 2 <= v <= m - sc.cpml - 2 for v, m in zip(p1, sc.n))
        h = ctypes.c_void_p()
        assert lib.fdtd_create_grid(*sc.n, sc.dx, sc.courant, None, None, ctypes.byref(h)) == 0
        try:
            for q0, q1, rr in sc.wires:
                assert lib.fdtd_add_wire(h, *q0, *q1, rr, None) == 0
            assert lib.fdtd_add_oblique_wire(h, *p0, *p1, r, None) == 0
            lim = ctypes.c_double()
            assert lib.fdtd_wire_courant_limit(h, ctypes.byref(lim)) == 0
            assert sc.courant < lim.value, (sc.name, lim.value)
        finally:
            lib.fdtd_destroy(h)
