"""Values the paper prints (tests/golden/, each file citing its source):
the four-term Debye expansions of its soil examples.  They pin the oracle's
dispersive media at the paper's own parameters -- four poles whose time
constants span three decades, deps up to 839 -- against the exact solution
of the continuous equations (CPU only; nothing here comes from the CUDA
library)."""
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle.oracle import EX, EY, EZ, HX, HY, HZ, OracleGrid
from paper_2207_06908_gb300 import workloads as W
from test_debye_pins import relaxation_matrix
from test_oracle_pins import grad_fields, node_potential

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "debye_tables.txt")


def debye_tables():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, *v = line.split()
                v = [float(x) for x in v]
                rows[name] = dict(rho0=v[0], sigma0=v[1], eps_inf=v[2], deps=v[3::2], tau=v[4::2])
    return rows


def test_printed_tables_are_transcribed_consistently():
    """each printed row pairs rho_0 with sigma_0 = 1 / rho_0 (to the printed
    digits) and has four poles"""
    rows = debye_tables()
    assert set(rows) == {"measured_soil", "layer_200", "layer_400", "layer_800"}
    for r in rows.values():
        assert abs(r["sigma0"] * r["rho0"] - 1.0) < 5e-4
        assert len(r["deps"]) == len(r["tau"]) == 4


def test_workloads_use_the_printed_parameters():
    rows = debye_tables()
    s = rows["measured_soil"]
    assert W.PAPER_SOIL["eps_inf"] == s["eps_inf"] and W.PAPER_SOIL["sigma"] == s["sigma0"]
    assert list(W.PAPER_SOIL["deps"]) == s["deps"] and list(W.PAPER_SOIL["tau"]) == s["tau"]
    for (eps_inf, sigma, deps, tau), name in zip(W.PAPER_LAYERS, ("layer_200", "layer_400", "layer_800")):
        r = rows[name]
        assert (eps_inf, sigma, list(deps), list(tau)) == (r["eps_inf"], r["sigma0"], r["deps"], r["tau"])


def relaxation_error(p, courant, t_start, t_run):
    """a curl-free E in a uniform soil of parameters p: the oracle's leapfrog
    (ADE) against the exact solution of the continuous relaxation equations
    from t_start to t_start + t_run; relative max error of E, max |H|, and
    the exact amplitude at the end"""
    rng = np.random.default_rng(12)
    n, dx = (7, 6, 8), 0.5
    g = OracleGrid(*n, dx, courant=courant)
    g.set_materials(np.zeros((n[2], n[1], n[0]), np.uint8), [p["eps_inf"]], [p["sigma0"]], [1.0])
    g.set_debye(0, p["deps"], p["tau"])
    g.finalize()
    steps = int(round(t_run / g.dt))
    ex, ey, ez = grad_fields(node_potential(rng, n), dx)
    A = relaxation_matrix(p["eps_inf"], p["sigma0"], p["deps"], p["tau"])
    x0 = np.zeros(A.shape[0])
    x0[0] = 1.0
    xs = expm(A * t_start) @ x0
    for c, v in ((EX, ex), (EY, ey), (EZ, ez)):
        g.set_field(c, xs[0] * v)
        for q in range(4):
            g.set_debye_current(c, q, xs[1 + q] * v)
    g.step(steps)
    x = expm(A * (t_start + steps * g.dt)) @ x0
    err = max(np.max(np.abs(g.get_field(c) - x[0] * v)) / np.max(np.abs(v))
              for c, v in ((EX, ex), (EY, ey), (EZ, ez)))
    h = max(np.max(np.abs(g.get_field(c))) for c in (HX, HY, HZ))
    return err, h, x[0]


@pytest.mark.parametrize("name", ["measured_soil", "layer_200", "layer_800"])
def test_oracle_relaxes_the_printed_soils_exactly_to_second_order(name):
    """E decays through conduction and four polarisation currents; the
    oracle's error falls as dt^2 towards the exact continuous solution (a
    wrong pole weight, time constant or sign fails at once)"""
    p = debye_tables()[name]
    e1, h1, amp = relaxation_error(p, 0.99, 2.0e-8, 1.5e-7)
    e2, h2, _ = relaxation_error(p, 0.495, 2.0e-8, 1.5e-7)
    assert h1 <= 1e-12 and h2 <= 1e-12
    assert 0.02 < abs(amp) < 0.9                  # well under way
    assert e1 <= 1e-5
    assert 3.6 <= e1 / e2 <= 4.4
