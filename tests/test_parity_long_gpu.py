"""GPU (FP32, through the C ABI) against the FP64 oracle at the step counts
the workloads state, from rest, at full size and in the launch shape the
benchmark times: the Sec. 2.1 leapfrog (Eq. fdtdhx, fdtdex) with the Sec. 2.2
CPML, the Sec. 2.3 thin wires and the Sec. 4 sources and probes, iterated for
the workload's whole run.

Bars: fields max(1e-5, 2x the error of the same algorithm evaluated with
FP32 storage), probes max(1e-4, 2x that error of the probe), the from-rest
reading: a source's near field is orders of magnitude above the field left
at the end, and a quasi-static H built from thousands of small increments
carries their FP32 rounding, so any FP32 field store costs more than the
stated bars on some quantities (the H fields after 4000 steps of the 256^3
workload: 2.6e-5; the wire current one cell below the wire's open top, a
small signal: 1.5e-4).  Every error
achieved is recorded beside both bars (FDTD_PARITY_RECORD, see
tests/parity_summary.py).

Oracle time on 16 host cores: about 3 min for the 256^3 run (FP64 and the
FP32 yardstick), 2 min for the 512x512x384 run.
"""
import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W
from _scenario import COMPONENTS, field_errors, oracle_from_scenario, record, rel_l2

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-5
PROBE_TOL = 1e-4


@pytest.fixture(scope="module")
def fdtd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd as F
    return F


def gpu_results(g, n_probes, steps):
    return [g.get_field(c) for c in range(6)], [g.read_probe(p, 0, steps) for p in range(n_probes)]


def oracle_results(sc, steps, f32=False):
    from oracle.oracle import OracleGrid
    o = OracleGrid.from_scenario(sc, parity=True, f32=f32)
    o.step(steps)
    out = [o.get_field(c) for c in range(6)], [o.read_probe(p)[:steps] for p in range(len(sc.probes))]
    del o
    return out


def check_from_rest(case, sc, steps, gf, gp):
    """oracle in FP64, then the FP32-storage yardstick; record and assert"""
    of, op = oracle_results(sc, steps)
    yf, yp = oracle_results(sc, steps, f32=True)
    fails = []
    for c, ((e, norm), (yard, _)) in enumerate(zip(field_errors(gf, of), field_errors(yf, of))):
        bar = max(FIELD_TOL, 2.0 * yard)
        record(case, f"field {COMPONENTS[c]}", e, bar, fp32_yardstick=yard, steps=steps, norm=norm)
        if not e <= bar:
            fails.append(f"{COMPONENTS[c]}: {e:.3e} > {bar:.3e}")
    for p in range(len(gp)):
        assert np.linalg.norm(op[p]) > 0, f"probe {p} saw nothing"
        e = rel_l2(gp[p], op[p])
        yard = rel_l2(yp[p], op[p])
        bar = max(PROBE_TOL, 2.0 * yard)
        record(case, f"probe {p}", e, bar, fp32_yardstick=yard, steps=steps)
        if not e <= bar:
            fails.append(f"probe {p}: {e:.3e} > {bar:.3e}")
    assert not fails, f"{case}: " + "; ".join(fails)


def test_config2_full_4000_steps_from_rest(fdtd):
    """256^3, 10-cell CPML, soil half-space, the 30 m thin wire fed by the
    1.2/50 us 10 kA double exponential, six probes: all 4000 steps of the
    workload (3.8 us; the front crosses the CPML and the wire top), stepped
    as the benchmark steps it (32-step graphs)"""
    steps = 4000
    sc = W.config2(n_steps=steps)
    g = fdtd.from_scenario(sc, probe_capacity=steps)
    g.step(steps)
    gf, gp = gpu_results(g, len(sc.probes), steps)
    g.close()
    check_from_rest("config2 256^3 CPML10 wire", sc, steps, gf, gp)


def test_config3_full_size_with_source_from_rest(fdtd):
    """512x512x384, 12-cell CPML, two-layer soil, the buried 8x8 mesh with its
    down-conductor and leads, driven by its 1 kA / 0.5 us ramp: 400 steps
    from rest at full size (the ramp reaches 380 A; the front has crossed
    the mesh and reached the CPML above the source)"""
    steps = 400
    sc = W.config3(n_steps=steps)
    g = fdtd.from_scenario(sc, probe_capacity=steps)
    g.step(steps)
    gf, gp = gpu_results(g, len(sc.probes), steps)
    g.close()
    check_from_rest("config3 512x512x384 CPML12 mesh", sc, steps, gf, gp)


def test_config4_smallest_and_largest_domain_2000_steps(fdtd):
    """the whole batched workload (256 grounding domains, sides 48..128,
    8-cell CPML) in the benchmark's launch shape (tuned tile depth per size
    class) for all 2000 steps from rest; the smallest and the largest domain
    against the oracle: fields and both probes (gap voltage, source current)"""
    from paper_2207_06908_gb300 import grounding
    steps = W.GROUND_STEPS
    scs = W.config4(n_steps=steps)
    sizes = [sc.n[0] for sc in scs]
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes))]
    blocks = {}
    for sc in scs:
        c = grounding.size_class(sc.n[0])
        if c not in blocks:
            blocks[c] = grounding.tune_block(sc.n[0])
    grids = [fdtd.from_scenario(sc, probe_capacity=steps, block=blocks[grounding.size_class(sc.n[0])])
             for sc in scs]
    b = fdtd.Batch(grids)
    b.step(steps)
    b.synchronize()
    got = {q: gpu_results(grids[q], len(scs[q].probes), steps) for q in picks}
    b.close()
    for g in grids:
        g.close()
    for q in picks:
        sc = scs[q]
        check_from_rest(f"config4 domain {q} ({sc.n[0]}^3) in the 256-domain batch", sc, steps, *got[q])
