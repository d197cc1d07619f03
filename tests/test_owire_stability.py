"""Stability bound of oblique thin wires (CPU): the Courant limit the
library enforces (fdtd_wire_courant_limit, host only) keeps the coupled
leapfrog of the FP64 oracle bounded over long runs for the stiffest
coupling (thick wires along node lines) and for a thick inclined tower, and
the limit is not vacuous: a few percent above it the same runs grow."""
import ctypes
import math

import numpy as np
import pytest

from oracle.oracle import OracleGrid
from test_oracle_pins import random_fields

R0 = math.exp(-0.57721566490153286) / (2 * math.sqrt(2))


def library_limit(n, dx, wires):
    from paper_2207_06908_gb300 import _lib as L
    lib = L.load()
    h = ctypes.c_void_p()
    assert lib.fdtd_create_grid(*n, dx, 0.5, None, None, ctypes.byref(h)) == 0
    try:
        for p0, p1, r in wires:
            assert lib.fdtd_add_oblique_wire(h, *map(float, p0), *map(float, p1), float(r), None) == 0
        c = ctypes.c_double()
        assert lib.fdtd_wire_courant_limit(h, ctypes.byref(c)) == 0
        return c.value
    finally:
        lib.fdtd_destroy(h)


def growth(n, dx, wires, S, steps=8000, seed=0):
    g = OracleGrid(*n, dx, courant=S, parity=False)
    for p0, p1, r in wires:
        g.add_oblique_wire(p0, p1, r)
    g.finalize()
    rng = np.random.default_rng(seed)
    f = random_fields(rng, n)
    for c in range(6):
        g.set_field(c, f[c])
    ns, nn = g.wire_counts()
    g.set_wire_state(rng.standard_normal(ns) * 0.01, rng.standard_normal(nn) * 1e-13)
    e0 = max(float(np.abs(g.get_field(c)).max()) for c in range(3))
    g.step(steps)
    e1 = max(float(np.abs(g.get_field(c)).max()) for c in range(3))
    return e1 / e0 if np.isfinite(e1) else math.inf


def node_line_wires(lam, dx):
    a = dx * R0 / math.exp(lam)
    return [((1.0, 7.0, 7.0), (13.0, 7.0, 7.0), a), ((7.0, 1.0, 3.0), (7.0, 13.0, 3.0), a),
            ((3.0, 3.0, 1.0), (3.0, 3.0, 13.0), a)]


@pytest.mark.parametrize("lam", [0.7, 1.3, 2.0])
def test_bound_holds_for_wires_along_node_lines(lam):
    n, dx = (14, 14, 14), 0.1
    wires = node_line_wires(lam, dx)
    lim = library_limit(n, dx, wires)
    expect = 1 / math.sqrt(1 + 2.0 * math.exp(-1.89 * lam))
    assert abs(lim - expect) < 1e-9
    assert growth(n, dx, wires, lim) < 100


@pytest.mark.parametrize("lam", [0.7, 1.0])
def test_bound_is_close_to_the_real_limit(lam):
    n, dx = (14, 14, 14), 0.1
    wires = node_line_wires(lam, dx)
    lim = library_limit(n, dx, wires)
    assert growth(n, dx, wires, lim + 0.04) > 1e3


def test_bound_holds_for_a_thick_inclined_tower():
    n, dx = (30, 30, 30), 0.5
    top = (15.0, 15.0, 24.0)
    wires = [((10.3, 10.1, 12.0), top, 0.02), ((19.7, 10.2, 12.0), top, 0.02), ((19.6, 19.9, 12.0), top, 0.02),
             ((10.4, 19.8, 12.0), top, 0.02), (top, (15.0, 15.0, 27.0), 0.02)]
    lim = library_limit(n, dx, wires)
    assert lim < 0.99
    assert growth(n, dx, wires, lim, steps=6000) < 100
