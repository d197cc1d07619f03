"""Staircase (oblique) thin wires and multiwire junctions on the GPU against
the FP64 oracle: three oblique wires meeting at one node, a source on one
of them, CPML."""
import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W
from _scenario import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd as F
    return F


def star(steps, fields=None):
    n = (34, 30, 32)
    cm = W.paint_blocks(n, [((0, 0, 0), (34, 30, 12), 1)])
    hub = (17, 15, 16)
    sc = W.Scenario("star", n, 0.05, 0.99, 5, cm, [(1.0, 0.0, 1.0), (9.0, 0.01, 1.0)], n_steps=steps)
    sc.wire_paths = [(hub, (7, 8, 8), 0.004), (hub, (27, 10, 24), 0.006), (hub, (12, 24, 26), 0.003),
                     ((8, 22, 9), (26, 21, 9), 0.005)]
    dt = W.time_step(0.05, 0.99)
    t = (np.arange(steps) + 0.5) * dt
    sc.sources = [((27, 10, 24), 2, np.exp(-((t - 25 * dt) / (7 * dt)) ** 2))]
    sc.probes = [(1, hub, 0, 1), (1, hub, 2, 1), (0, (7, 8, 8), 2, 2), (2, (20, 14, 18), 1, 1)]
    sc.fields = fields
    return sc


def compare(F, sc, steps, bar_from_rest):
    from oracle.oracle import OracleGrid
    g = F.from_scenario(sc, probe_capacity=steps)
    if sc.fields is not None:
        for c, f in enumerate(sc.fields):
            g.set_field(c, f)
    g.step(steps)
    gf, gp = [g.get_field(c) for c in range(6)], [g.read_probe(p, 0, steps) for p in range(len(sc.probes))]
    g.close()
    o = OracleGrid.from_scenario(sc, parity=True)
    o.step(steps)
    of, op = [o.get_field(c) for c in range(6)], [o.read_probe(p)[:steps] for p in range(len(sc.probes))]
    bars = [1e-5] * 6
    if bar_from_rest:
        y = OracleGrid.from_scenario(sc, parity=True, f32=True)
        y.step(steps)
        bars = [max(1e-5, 2.0 * rel_l2(y.get_field(c), of[c])) for c in range(6)]
    for c in range(6):
        assert rel_l2(gf[c], of[c]) <= bars[c], c
    for p in range(len(gp)):
        if np.linalg.norm(op[p]) > 0:
            assert rel_l2(gp[p], op[p]) <= 1e-4, p


def test_star_junction_from_rest(fdtd):
    compare(fdtd, star(400), 400, True)


def test_star_junction_random_fields(fdtd):
    sc = star(60)
    sc.fields = W.random_fields(np.random.default_rng(9), sc.n)
    sc.sources = []
    compare(fdtd, sc, 60, False)
