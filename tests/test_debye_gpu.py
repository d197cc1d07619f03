"""Debye media on the GPU (dispersive-media kernel, coefficient classes,
source correction) against the FP64 oracle (the paper's "Dispersive media"
subsection; ADE method of its references).  Fields within 1e-5, probes
within 1e-4 (relative L2), as for the non-dispersive path."""
import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W
from _scenario import COMPONENTS, field_errors, oracle_from_scenario, record, rel_l2

pytestmark = pytest.mark.gpu
FIELD_TOL, PROBE_TOL = 1e-5, 1e-4


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd as F
    return F


def run_gpu(F, sc, steps, split=None):
    g = F.from_scenario(sc, probe_capacity=steps)
    if sc.fields is not None:
        for c, f in enumerate(sc.fields):
            g.set_field(c, f)
    for n in (split or [steps]):
        g.step(n)
    out = [g.get_field(c) for c in range(6)], [g.read_probe(p, 0, steps) for p in range(len(sc.probes))]
    g.close()
    return out


def run_oracle(sc, steps):
    o = oracle_from_scenario(sc, parity=True)
    o.step(steps)
    return [o.get_field(c) for c in range(6)], [o.read_probe(p)[:steps] for p in range(len(sc.probes))]


def compare(gf, gp, of, op):
    for c in range(6):
        e = rel_l2(gf[c], of[c])
        assert e <= FIELD_TOL, f"component {c}: rel L2 {e:.3e}"
    for p in range(len(gp)):
        if np.linalg.norm(op[p]) == 0:
            assert np.all(gp[p] == 0)
            continue
        e = rel_l2(gp[p], op[p])
        assert e <= PROBE_TOL, f"probe {p}: rel L2 {e:.3e}"


@pytest.mark.parametrize("seed,n,cpml", [(41, (17, 17, 17), 0), (42, (23, 19, 21), 3), (43, (45, 21, 27), 4),
                                         (44, (33, 20, 9), 2)])
def test_random_debye_media(fdtd, seed, n, cpml):
    """random blocky media, two of them dispersive (1-4 poles), thin wires,
    sources, probes, CPML; random fields; 60 steps"""
    sc = W.with_random_debye(W.random_scenario(seed, n=n, cpml=cpml, n_steps=60), seed + 100)
    compare(*run_gpu(fdtd, sc, 60), *run_oracle(sc, 60))


def soil_block_with_source(n_steps):
    """a four-pole soil block holding a wire and a source edge (the current
    correction of a dispersive source edge), CPML, from rest"""
    n = (30, 26, 28)
    cm = W.paint_blocks(n, [((0, 0, 0), (30, 26, 16), 1)])
    dt = W.time_step(0.05, 0.99)
    t = (np.arange(n_steps) + 0.5) * dt
    cur = np.exp(-((t - 30 * dt) / (8 * dt)) ** 2)
    sc = W.Scenario("soil_source", n, 0.05, 0.99, 4, cm, [(1.0, 0.0, 1.0), (8.0, 0.01, 1.0)],
                    wires=[((15, 13, 6), (15, 13, 12), 0.004)],
                    sources=[((15, 13, 12), 2, cur)],
                    probes=[(0, (15, 13, 12), 2, 1), (1, (15, 13, 12), 2, 1), (2, (18, 13, 10), 2, 1)],
                    n_steps=n_steps)
    sc.debye = {1: ([30.0, 12.0, 5.0, 60.0], [2 * dt * 10, 2 * dt * 40, 2 * dt * 150, 2 * dt * 5])}
    return sc


def test_source_on_dispersive_edge(fdtd):
    """probes within 1e-4; fields within the from-rest bar (the 1 A source's
    near field against the field left after 300 steps: twice the error of
    the same algorithm in FP32 storage, floor 1e-5)"""
    from oracle.oracle import OracleGrid
    sc = soil_block_with_source(300)
    gf, gp = run_gpu(fdtd, sc, 300)
    of, op = run_oracle(sc, 300)
    y = OracleGrid.from_scenario(sc, parity=True, f32=True)
    y.step(300)
    for c in range(6):
        bar = max(FIELD_TOL, 2.0 * rel_l2(y.get_field(c), of[c]))
        assert rel_l2(gf[c], of[c]) <= bar, c
    for p in range(len(gp)):
        assert rel_l2(gp[p], op[p]) <= PROBE_TOL, p


def test_debye_graph_and_direct_paths_agree(fdtd):
    sc = W.with_random_debye(W.random_scenario(45, n=(40, 18, 33), cpml=4, n_steps=75), 7)
    a = run_gpu(fdtd, sc, 75)
    b = run_gpu(fdtd, sc, 75, split=[1, 2, 33, 7, 32])
    for x, y in zip(a[0] + a[1], b[0] + b[1]):
        assert np.array_equal(x, y)


def test_debye_no_alloc_path_matches(fdtd):
    sc = W.with_random_debye(W.random_scenario(46, n=(20, 13, 18), cpml=3, n_steps=40), 8)
    a = run_gpu(fdtd, sc, 40)
    g = fdtd.from_scenario(sc, probe_capacity=40)
    for c, f in enumerate(sc.fields):
        g.set_field(c, f)
    g.step_noalloc(40)
    g.synchronize()
    for c in range(6):
        assert np.array_equal(a[0][c], g.get_field(c))
    g.close()


def test_debye_checkpoint_resume(fdtd):
    sc = W.with_random_debye(W.random_scenario(47, n=(20, 13, 18), cpml=3, n_steps=50), 9)
    g = fdtd.from_scenario(sc, probe_capacity=50)
    for c, f in enumerate(sc.fields):
        g.set_field(c, f)
    g.step(21)
    st = g.save_state()
    g.step(29)
    ref = [g.get_field(c) for c in range(6)]
    h = fdtd.from_scenario(sc, probe_capacity=50)
    h.load_state(st)
    h.step(29)
    for c in range(6):
        assert np.array_equal(ref[c], h.get_field(c))
    g.close()
    h.close()


def test_batch_rejects_dispersive_grids(fdtd):
    sc = W.with_random_debye(W.random_scenario(48, n=(17, 17, 17), n_steps=4), 10)
    g = fdtd.from_scenario(sc, probe_capacity=4)
    with pytest.raises(fdtd.FdtdError):
        fdtd.Batch([g])
    g.close()


def test_debye_soil_full_size_random_fields_no_source(fdtd):
    """the 256^3 dispersive-soil workload (four-pole Debye soil of the paper's
    measured-soil table, CPML, thin wire, probes) at full size without its
    source, from seeded random fields: fields within 1e-5 after 24 steps"""
    sc = W.debye_soil(n_steps=24)
    sc.sources = []
    sc.fields = W.random_fields(np.random.default_rng(2027), sc.n)
    compare(*run_gpu(fdtd, sc, 24), *run_oracle(sc, 24))


def test_three_layer_electrode_array_from_rest(fdtd):
    """the paper's apparent-resistivity geometry: three four-pole Debye
    layers, four rods with current and voltage leads, CPML, driven by the
    model file's Heidler pulse (it starts at step 1941); 3000 steps from
    rest.  Probes within 1e-4; fields within the from-rest bar (twice the
    FP32-storage error of the same algorithm, floor 1e-5)"""
    from oracle.oracle import OracleGrid
    steps = 3000
    sc = W.three_layer_array(n_steps=steps)
    gf, gp = run_gpu(fdtd, sc, steps)
    of, op = run_oracle(sc, steps)
    assert np.abs(op[0]).max() > 0              # the far voltage gap has seen the field
    y = OracleGrid.from_scenario(sc, parity=True, f32=True)
    y.step(steps)
    case = "three-layer Debye array, Heidler source"
    fails = []
    yards = field_errors([y.get_field(c) for c in range(6)], of)
    for c, ((e, norm), (yard, _)) in enumerate(zip(field_errors(gf, of), yards)):
        bar = max(FIELD_TOL, 2.0 * yard)
        record(case, f"field {COMPONENTS[c]}", e, bar, fp32_yardstick=yard, steps=steps, norm=norm)
        if not e <= bar:
            fails.append((c, e, bar))
    for p in range(len(gp)):
        e = rel_l2(gp[p], op[p])
        yard = rel_l2(y.read_probe(p)[:steps], op[p])
        bar = max(PROBE_TOL, 2.0 * yard)
        record(case, f"probe {p}", e, bar, fp32_yardstick=yard, steps=steps)
        if not e <= bar:
            fails.append((f"probe {p}", e, bar))
    assert not fails, fails
