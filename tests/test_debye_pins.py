"""Pins of the oracle's Debye media (the paper's "Dispersive media"
subsection: multi-term Debye permittivity by the auxiliary differential
equation method of its references) against the exact solution of the
continuous equations and exact identities (CPU only).

The continuous equations, per pole p:
    eps0 eps_inf dE/dt + sigma E + sum_p J_p = curl H,
    tau_p dJ_p/dt + J_p = eps0 deps_p dE/dt,   mu0 dH/dt = -curl E.
For a field that stays in one spatial pattern these reduce to a small
linear ODE in the pattern's amplitudes, solved here exactly with a matrix
exponential; the oracle's leapfrog solution must converge to it at second
order in dt.  Nothing here comes from the CUDA library.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from oracle.oracle import C0, EPS0, MU0, EX, EY, EZ, HX, HY, HZ, OracleGrid
from test_oracle_pins import curl_e, grad_fields, mode_fields, node_potential

EPS_INF, SIGMA = 5.0, 0.01
DEPS, TAU = [10.0, 20.0], [1.0e-9, 4.0e-9]


def relaxation_matrix(eps_inf, sigma, deps, tau, kappa2=None):
    """d/dt of the amplitudes [e, (eta,) j_1 .. j_P] of the continuous
    equations; with kappa2 (the pattern's curl-curl eigenvalue) the H
    amplitude eta (H = eta curl E_pattern, mu0 eta' = -e) is included"""
    P = len(deps)
    wave = kappa2 is not None
    n = 1 + wave + P
    A = np.zeros((n, n))
    e0 = EPS0 * eps_inf
    # e' = (kappa2 eta - sigma e - sum j) / e0
    A[0, 0] = -sigma / e0
    if wave:
        A[0, 1] = kappa2 / e0
        A[1, 0] = -1.0 / MU0
    for p in range(P):
        A[0, 1 + wave + p] = -1.0 / e0
    # j_p' = (eps0 deps_p e' - j_p) / tau_p
    for p in range(P):
        r = 1 + wave + p
        A[r, :] = EPS0 * deps[p] * A[0, :] / tau[p]
        A[r, r] -= 1.0 / tau[p]
    return A


def uniform_debye_grid(n, dx, courant):
    g = OracleGrid(*n, dx, courant=courant)
    g.set_materials(np.zeros((n[2], n[1], n[0]), np.uint8), [EPS_INF], [SIGMA], [1.0])
    g.set_debye(0, DEPS, TAU)
    g.finalize()
    return g


T_START = 3.0e-9        # the runs start from the exact solution at this time (nonzero currents)


def curl_free_error(courant, steps_at_099):
    rng = np.random.default_rng(5)
    n, dx = (7, 6, 8), 0.05
    g = uniform_debye_grid(n, dx, courant)
    dt = g.dt
    steps = int(round(steps_at_099 * 0.99 / courant))
    ex, ey, ez = grad_fields(node_potential(rng, n), dx)
    A = relaxation_matrix(EPS_INF, SIGMA, DEPS, TAU)
    x0 = np.array([1.0, 0.0, 0.0])
    xs = expm(A * T_START) @ x0                 # E and J_p share the time levels t_n
    for c, v in ((EX, ex), (EY, ey), (EZ, ez)):
        g.set_field(c, xs[0] * v)
        for p in range(2):
            g.set_debye_current(c, p, xs[1 + p] * v)
    g.step(steps)
    x = expm(A * (T_START + steps * dt)) @ x0
    err = max(np.max(np.abs(g.get_field(c) - x[0] * v)) / np.max(np.abs(v))
              for c, v in ((EX, ex), (EY, ey), (EZ, ez)))
    h = max(np.max(np.abs(g.get_field(c))) for c in (HX, HY, HZ))
    return err, h, x[0]


def test_curl_free_relaxation_converges_to_exact_solution():
    """a curl-free E in a uniform two-pole Debye conductor never excites H;
    each edge follows e(t) of the continuous relaxation equations with an
    error that falls as dt^2"""
    e1, h1, amp = curl_free_error(0.99, 90)
    e2, h2, _ = curl_free_error(0.495, 90)
    assert h1 <= 1e-14 and h2 <= 1e-14          # E is O(10); curl of a gradient is rounding only
    assert 0.05 < amp < 0.95                    # the relaxation is well under way
    assert e1 <= 1e-6
    assert 3.3 <= e1 / e2 <= 4.8                # second order


def cavity_error(courant, steps_at_099):
    n, dx, m = (12, 10, 8), 0.05, (1, 1, 0)
    g = uniform_debye_grid(n, dx, courant)
    dt = g.dt
    steps = int(round(steps_at_099 * 0.99 / courant))
    ex, ey, ez, kk = mode_fields(n, dx, m, (0.0, 0.0, 1.0))
    cx, cy, cz = curl_e(ex, ey, ez, dx)
    kappa2 = sum((2.0 * math.sin(k * dx / 2) / dx) ** 2 for k in kk)
    A = relaxation_matrix(EPS_INF, SIGMA, DEPS, TAU, kappa2)
    x0 = np.array([1.0, 0.0, 0.0, 0.0])
    xs = expm(A * T_START) @ x0                 # E and J_p at t = T_START
    xh = expm(A * (T_START - dt / 2)) @ x0      # H half a step earlier
    for c, v in ((EX, ex), (EY, ey), (EZ, ez)):
        g.set_field(c, xs[0] * v)
        for p in range(2):
            g.set_debye_current(c, p, xs[2 + p] * v)
    for c, v in ((HX, cx), (HY, cy), (HZ, cz)):
        g.set_field(c, xh[1] * v)
    g.step(steps)
    x = expm(A * (T_START + steps * dt)) @ x0
    ref = x[0] * ez
    return np.linalg.norm(g.get_field(EZ) - ref) / np.linalg.norm(ez), x[0]


def test_cavity_mode_in_debye_medium_converges_to_exact_solution():
    """the TM110 mode of a PEC box filled with a two-pole Debye conductor:
    E, H and both polarisation currents keep the mode's shape, and its
    amplitude follows the continuous equations (curl coupling, loss and
    relaxation together) with an error that falls as dt^2"""
    e1, amp = cavity_error(0.99, 40)
    e2, _ = cavity_error(0.495, 40)
    assert abs(amp) > 0.1                       # still oscillating, damped
    assert e1 <= 3e-4
    assert 3.3 <= e1 / e2 <= 4.8


def random_media_grid(rng, n, debye, courant=0.99):
    g = OracleGrid(*n, 0.05, courant=courant)
    cm = rng.integers(0, 3, (n[2], n[1], n[0])).astype(np.uint8)
    g.set_materials(cm, [3.0, 9.0, 15.0], [0.0, 0.02, 0.005], [1.0, 1.0, 2.0])
    for mat, (d, t) in debye.items():
        g.set_debye(mat, d, t)
    g.finalize()
    f = [rng.standard_normal((n[2], n[1], n[0])) for _ in range(6)]
    for c in range(6):
        g.set_field(c, f[c] * (1.0 if c < 3 else 1.0 / 377.0))
    return g


def test_equal_tau_poles_add_up():
    """two poles with one tau act as a single pole with the summed deps
    (the sum over poles): fields agree to rounding after 80 steps of random
    fields in random media, where one material is dispersive (edges average
    each pole over their cells)"""
    n = (9, 8, 7)
    a = random_media_grid(np.random.default_rng(1), n, {1: ([4.0, 6.0], [2e-9, 2e-9])})
    b = random_media_grid(np.random.default_rng(1), n, {1: ([10.0], [2e-9])})
    a.step(80)
    b.step(80)
    for c in range(6):
        fa, fb = a.get_field(c), b.get_field(c)
        assert np.max(np.abs(fa - fb)) <= 1e-11 * np.max(np.abs(fb))
    ja = a.get_debye_current(EZ, 0) + a.get_debye_current(EZ, 1)
    jb = b.get_debye_current(EZ, 0)
    assert np.max(np.abs(ja - jb)) <= 1e-11 * np.max(np.abs(jb))
    assert np.max(np.abs(jb)) > 0


def test_absent_debye_material_changes_nothing():
    """poles on a material no cell uses: every edge keeps the
    non-dispersive update, bit for bit"""
    n = (8, 9, 7)
    a = random_media_grid(np.random.default_rng(2), n, {7: ([5.0, 1.0], [1e-9, 1e-8])})
    b = random_media_grid(np.random.default_rng(2), n, {})
    a.step(50)
    b.step(50)
    for c in range(6):
        assert np.array_equal(a.get_field(c), b.get_field(c))


def test_dispersion_changes_the_fields():
    """the same run with and without poles on a used material differs (the
    Debye terms are applied), and stays bounded over 2000 steps"""
    n = (8, 9, 7)
    a = random_media_grid(np.random.default_rng(3), n, {1: ([30.0, 80.0], [3e-10, 3e-9])})
    b = random_media_grid(np.random.default_rng(3), n, {})
    a.step(40)
    b.step(40)
    assert np.max(np.abs(a.get_field(EX) - b.get_field(EX))) > 1e-3
    a.step(1960)
    assert all(np.isfinite(a.get_field(c)).all() and np.max(np.abs(a.get_field(c))) < 1e3 for c in range(6))


def wire_run(radius, steps, src=True):
    n, dx = (14, 12, 16), 0.05
    g = OracleGrid(*n, dx)
    cm = np.zeros((n[2], n[1], n[0]), np.uint8)
    cm[:8] = 1
    g.set_materials(cm, [1.0, 12.0], [0.0, 0.004], [1.0, 1.0])
    g.set_debye(1, [40.0, 15.0], [2e-9, 3e-8])
    if radius is not None:
        g.add_wire((7, 6, 3), (7, 6, 12), radius)
    if src:
        dt = g.dt
        t = (np.arange(steps) + 0.5) * dt
        g.add_source((7, 6, 12), 2, np.exp(-((t - 40 * dt) / (12 * dt)) ** 2))
    g.add_probe(0, (7, 6, 12), 2, 1)
    g.finalize(steps)
    g.step(steps)
    return g


def test_wire_r0_in_debye_medium_equals_pec_edge():
    """m = 1 (a = 0.23 dx) leaves every coefficient of the dispersive soil
    unscaled (ca and cb of a Debye edge contain sum beta_p, so they would
    move with deps): the wire is exactly a line of PEC edges"""
    c0 = wire_run(None, 0, src=False)
    c1 = wire_run(0.23 * 0.05, 0, src=False)
    for w in range(9):
        d = c0.get_coef(w) != c1.get_coef(w)
        if w in (2, 5):                         # ca_z, cb_z: the nine on-wire Ez edges, now PEC
            assert d.sum() == 9 and np.all(c1.get_coef(w)[d] == 0)
        else:
            assert not d.any()
    # a thinner wire does scale them: cb of the 20 radial Ex edges (ca is a
    # ratio of terms that all scale with m)
    c2 = wire_run(0.004, 0, src=False)
    assert (c0.get_coef(3) != c2.get_coef(3)).sum() == 20


def test_thin_wire_in_debye_medium_is_stable():
    """a thin wire (m < 1, every deps scaled by m with eps and sigma) in the
    two-pole soil, driven by a pulse: bounded after 3000 steps"""
    g = wire_run(0.004, 3000)
    v = g.read_probe(0)
    assert np.all(np.isfinite(v)) and np.abs(v[-500:]).max() < np.abs(v).max()
    for c in range(6):
        assert np.isfinite(g.get_field(c)).all()
