"""Pins of the oracle's lumped elements and non-ideal / voltage sources (the
paper's sources and lumped circuit elements, in the forms of the textbook it
cites) against circuit laws: Ohm's law and Kirchhoff's voltage law in a
wire loop, a capacitor's charging slope, a voltage divider, plus exact
identities (CPU only)."""
import numpy as np
import pytest

from oracle.oracle import EPS0, EX, EY, EZ, OracleGrid
from paper_2207_06908_gb300 import workloads as W

DX = 0.05


def loop_grid(steps, gap_left, gap_right, i0=1.0, rise=400):
    """a PEC box 20 x 16 x 20 cells with a square wire loop (x = 6..14,
    z = 6..14 at y = 8, r = 5 mm) cut by one-cell gaps on its left and right
    sides at z = 10; gap_left / gap_right: callables that install the
    element of that gap on the grid"""
    g = OracleGrid(20, 16, 20, DX)
    g.set_materials(np.zeros((20, 16, 20), np.uint8), [1.0], [0.0], [1.0])
    r = 0.005
    for p0, p1 in [((6, 8, 6), (14, 8, 6)), ((6, 8, 14), (14, 8, 14)), ((6, 8, 6), (6, 8, 10)),
                   ((6, 8, 11), (6, 8, 14)), ((14, 8, 6), (14, 8, 10)), ((14, 8, 11), (14, 8, 14))]:
        g.add_wire(p0, p1, r)
    gap_left(g, (6, 8, 10))
    gap_right(g, (14, 8, 10))
    g.add_probe(0, (6, 8, 10), 2, 1)
    g.add_probe(0, (14, 8, 10), 2, 1)
    g.finalize(steps)
    return g


def current_ramp(g, steps, i0=1.0, rise=400):
    n = np.arange(steps)
    return i0 * np.minimum((n + 0.5) / rise, 1.0)


def test_resistor_ohm_and_kirchhoff():
    """a 1 A current source driving a 20 ohm resistor round a wire loop: once
    the L/R transient has passed, the resistor's voltage is I R (Ohm) and, by
    Kirchhoff's voltage law (no flux change), the source gap's equals it (both
    gaps measured along +z, traversed in opposite senses round the loop)"""
    steps, R = 4000, 20.0
    g = loop_grid(steps, lambda g, p: g.add_source(p, 2, current_ramp(g, steps)),
                  lambda g, p: g.add_lumped(p, 2, resistance=R))
    g.step(steps)
    vs, vr = g.read_probe(0)[-300:].mean(), g.read_probe(1)[-300:].mean()
    # current up the left side, down the right: V = -E dx across the resistor is +I R
    assert abs(vr - R) <= 0.02 * R
    assert abs(vs - R) <= 0.02 * R


def test_capacitor_charging_slope():
    """the same loop closed by a 1 nF capacitor: after the ramp the voltage
    grows as I t / C (the loop's own stray capacitance, about 7 pF, stays
    under 1%)"""
    steps, C = 3000, 1e-9
    g = loop_grid(steps, lambda g, p: g.add_source(p, 2, current_ramp(g, steps)),
                  lambda g, p: g.add_lumped(p, 2, capacitance=C))
    g.step(steps)
    v = g.read_probe(1)
    n1, n2 = 1500, 2900
    slope = (v[n2] - v[n1]) / ((n2 - n1) * g.dt)
    assert abs(slope - 1.0 / C) <= 0.02 / C


def test_thevenin_source_voltage_divider():
    """a 10 V source with 30 ohm internal resistance into a 70 ohm load:
    7 V across the load and the source terminals at steady state"""
    steps = 4000
    v = np.minimum((np.arange(steps) + 0.5) / 400.0, 1.0) * 10.0
    g = loop_grid(steps, lambda g, p: g.add_voltage_source(p, 2, v, r_internal=30.0),
                  lambda g, p: g.add_lumped(p, 2, resistance=70.0))
    g.step(steps)
    vs, vl = g.read_probe(0)[-300:].mean(), g.read_probe(1)[-300:].mean()
    # terminal voltage 10 - 30 I with I = 0.1 A; both gaps read it (KVL, as above)
    assert abs(vs - 7.0) <= 0.02 * 7.0
    assert abs(vl - 7.0) <= 0.02 * 7.0


def test_norton_source_parallel_resistance():
    """1 A with 50 ohm in parallel into a 50 ohm load: half the current
    flows in the load, 25 V across it"""
    steps = 4000
    g = loop_grid(steps, lambda g, p: g.add_source(p, 2, current_ramp(g, steps), r_internal=50.0),
                  lambda g, p: g.add_lumped(p, 2, resistance=50.0))
    g.step(steps)
    vl = g.read_probe(1)[-300:].mean()
    assert abs(vl - 25.0) <= 0.02 * 25.0


def test_ideal_voltage_source_fixes_gap_voltage():
    """an ideal voltage source makes the gap voltage exactly V(t_{n+1})"""
    steps = 300
    v = np.sin(np.arange(steps) * 0.05) * 3.0
    g = loop_grid(steps, lambda g, p: g.add_voltage_source(p, 2, v),
                  lambda g, p: g.add_lumped(p, 2, resistance=50.0))
    g.step(steps)
    np.testing.assert_allclose(g.read_probe(0), v, rtol=0, atol=1e-14)


def uniform_run(lumped=None, sigma=0.0, eps_r=1.0, steps=60):
    rng = np.random.default_rng(4)
    n = (8, 7, 9)
    g = OracleGrid(*n, DX)
    g.set_materials(np.zeros((n[2], n[1], n[0]), np.uint8), [eps_r], [sigma], [1.0])
    if lumped:
        for axis in range(3):
            for k in range(n[2]):
                for j in range(n[1]):
                    for i in range(n[0]):
                        p = [i, j, k]
                        if all((0 <= p[u] < n[u]) if u == axis else (1 <= p[u] <= n[u] - 1) for u in range(3)):
                            g.add_lumped(tuple(p), axis, *lumped)
    g.finalize()
    for c in range(6):
        g.set_field(c, rng.standard_normal((n[2], n[1], n[0])) * (1.0 if c < 3 else 1 / 377))
    g.step(steps)
    return [g.get_field(c) for c in range(6)]


def test_lumped_elements_on_every_edge_equal_a_medium():
    """a resistor R on every interior E edge is the conductivity 1/(R dx);
    a capacitor C on every edge adds the permittivity C/dx (identical
    updates: bit for bit for R, to rounding for C)"""
    R, C = 40.0, 3e-12
    a, b = uniform_run(lumped=(R, 0.0)), uniform_run(sigma=1.0 / (R * DX))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    a, b = uniform_run(lumped=(0.0, C)), uniform_run(eps_r=1.0 + C / (DX * EPS0))
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) <= 1e-12 * np.max(np.abs(y))


def test_heidler_peak_and_shape():
    """the Heidler function with its peak correction peaks at i0 to within
    the correction's accuracy, rises as (t/tau1)^n and decays as exp(-t/tau2)"""
    for i0, t1, t2, n in [(1.0, 3.7e-7, 1.4e-5, 10), (10e3, 19e-6, 485e-6, 10), (1.0, 0.25e-6, 100e-6, 10)]:
        t = np.linspace(0, 10 * t1 + 3 * t2, 400001)
        i = W.heidler(t, i0, t1, t2, n)
        assert abs(i.max() - i0) <= 0.02 * i0
        assert i[0] == 0.0
        late = t > 20 * t1
        ratio = i[late][1:] / i[late][:-1]
        assert np.allclose(ratio, np.exp(-(t[1] - t[0]) / t2), rtol=1e-3)
