"""Lumped resistors / capacitors, non-ideal current sources and voltage
sources on the GPU (coefficient classes and the source kernel) against the
FP64 oracle.  Probes within 1e-4; fields within 1e-5 for random fields,
within the from-rest bar for source-driven runs from rest."""
import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W
from _scenario import oracle_from_scenario, rel_l2

pytestmark = pytest.mark.gpu
FIELD_TOL, PROBE_TOL = 1e-5, 1e-4


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd as F
    return F


def run_gpu(F, sc, steps):
    g = F.from_scenario(sc, probe_capacity=steps)
    if sc.fields is not None:
        for c, f in enumerate(sc.fields):
            g.set_field(c, f)
    g.step(steps)
    out = [g.get_field(c) for c in range(6)], [g.read_probe(p, 0, steps) for p in range(len(sc.probes))]
    g.close()
    return out


def run_oracle(sc, steps, f32=False):
    from oracle.oracle import OracleGrid
    o = OracleGrid.from_scenario(sc, parity=True, f32=f32)
    o.step(steps)
    return [o.get_field(c) for c in range(6)], [o.read_probe(p)[:steps] for p in range(len(sc.probes))]


def check(F, sc, steps, from_rest):
    gf, gp = run_gpu(F, sc, steps)
    of, op = run_oracle(sc, steps)
    if from_rest:
        yf, _ = run_oracle(sc, steps, f32=True)
    for c in range(6):
        bar = max(FIELD_TOL, 2.0 * rel_l2(yf[c], of[c])) if from_rest else FIELD_TOL
        assert rel_l2(gf[c], of[c]) <= bar, c
    for p in range(len(gp)):
        if np.linalg.norm(op[p]) == 0:
            assert np.all(gp[p] == 0)
        else:
            assert rel_l2(gp[p], op[p]) <= PROBE_TOL, p


def loop(steps, left, right, debye=False):
    """the wire loop of the oracle's circuit pins: PEC box 20 x 16 x 20
    cells, square loop at y = 8 with gaps on both sides at z = 10"""
    n = (20, 16, 20)
    cm = np.zeros((20, 16, 20), np.uint8)
    if debye:
        cm[:11] = 1
    r = 0.005
    wires = [((6, 8, 6), (14, 8, 6), r), ((6, 8, 14), (14, 8, 14), r), ((6, 8, 6), (6, 8, 10), r),
             ((6, 8, 11), (6, 8, 14), r), ((14, 8, 6), (14, 8, 10), r), ((14, 8, 11), (14, 8, 14), r)]
    sc = W.Scenario("loop", n, 0.05, 0.99, 0, cm, [(1.0, 0.0, 1.0), (6.0, 0.003, 1.0)], wires=wires,
                    probes=[(0, (6, 8, 10), 2, 1), (0, (14, 8, 10), 2, 1), (1, (6, 8, 10), 2, 1)], n_steps=steps)
    left(sc, (6, 8, 10))
    right(sc, (14, 8, 10))
    if debye:
        sc.debye = {1: ([20.0, 8.0], [3e-9, 2e-8])}
    return sc


def ramp(steps, top, rise=300):
    return top * np.minimum((np.arange(steps) + 0.5) / rise, 1.0)


@pytest.mark.parametrize("case", ["resistor", "capacitor", "thevenin", "norton", "ideal_v", "ideal_v_debye"])
def test_loop_circuits_match_oracle(fdtd, case):
    steps = 1200
    src = {"resistor": lambda sc, p: sc.sources.append((p, 2, ramp(steps, 1.0))),
           "capacitor": lambda sc, p: sc.sources.append((p, 2, ramp(steps, 1.0))),
           "thevenin": lambda sc, p: sc.vsources.append((p, 2, ramp(steps, 10.0), 30.0)),
           "norton": lambda sc, p: sc.sources.append((p, 2, ramp(steps, 1.0), 50.0)),
           "ideal_v": lambda sc, p: sc.vsources.append((p, 2, np.sin(np.arange(steps) * 0.03) * 3.0, 0.0)),
           "ideal_v_debye": lambda sc, p: sc.vsources.append((p, 2, np.sin(np.arange(steps) * 0.03) * 3.0, 0.0))}[case]
    load = {"capacitor": lambda sc, p: sc.lumped.append((p, 2, 0.0, 1e-9))}.get(
        case, lambda sc, p: sc.lumped.append((p, 2, 20.0 if case == "resistor" else 70.0, 0.0)))
    sc = loop(steps, src, load, debye=case.endswith("debye"))
    check(fdtd, sc, steps, from_rest=True)


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_random_lumped_elements_and_sources(fdtd, seed):
    """random media (two dispersive), wires, CPML, random fields, plus random
    lumped R / C / RC elements, non-ideal current sources and ideal /
    series-resistance voltage sources on random interior edges; 50 steps"""
    rng = np.random.default_rng(seed)
    n = (23, 19, 21)
    sc = W.with_random_debye(W.random_scenario(seed, n=n, cpml=3, n_steps=50), seed + 7)
    lo = 4

    def edge():
        axis = int(rng.integers(0, 3))
        return tuple(int(rng.integers(lo, m - lo)) for m in n), axis

    for _ in range(6):
        node, axis = edge()
        r = float(10 ** rng.uniform(0, 3)) if rng.random() < 0.7 else 0.0
        c = float(10 ** rng.uniform(-13, -10)) if (r == 0.0 or rng.random() < 0.4) else 0.0
        sc.lumped.append((node, axis, r, c))
    t = np.arange(50)
    for q in range(3):
        node, axis = edge()
        sc.sources.append((node, axis, np.sin(0.2 * t + q), float(10 ** rng.uniform(1, 3))))
    for q in range(3):
        node, axis = edge()
        sc.vsources.append((node, axis, 2.0 * np.cos(0.15 * t + q), 0.0 if q == 0 else float(10 ** rng.uniform(1, 3))))
    check(fdtd, sc, 50, from_rest=False)
