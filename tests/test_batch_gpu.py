"""Batched engine: many independent domains advanced by one persistent launch
per step.  It must give exactly the results of stepping each grid alone, and
match the FP64 oracle on grounding domains of the batched workload's shape."""
import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W
from _scenario import oracle_from_scenario, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdtd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd as F
    return F


def build(F, sc, steps):
    g = F.from_scenario(sc, probe_capacity=steps)
    if sc.fields is not None:
        for c, f in enumerate(sc.fields):
            g.set_field(c, f)
    return g


def test_batch_equals_individual_grids(fdtd):
    """uneven sizes, with and without CPML, wires, sources, probes; 45 steps
    (one 32-step graph + direct launches): bitwise equal to fdtd_step"""
    scs = [W.random_scenario(200 + q, n=n, cpml=c, n_steps=45)
           for q, (n, c) in enumerate([((17, 17, 17), 0), ((45, 21, 27), 5), ((33, 40, 18), 3),
                                       ((64, 16, 30), 0), ((20, 35, 41), 4)])]
    steps = 45
    alone = []
    for sc in scs:
        g = build(fdtd, sc, steps)
        g.step(steps)
        alone.append(([g.get_field(c) for c in range(6)], [g.read_probe(p) for p in range(len(sc.probes))]))
        g.close()
    grids = [build(fdtd, sc, steps) for sc in scs]
    b = fdtd.Batch(grids)
    b.step(steps)
    b.synchronize()
    for g, sc, (fa, pa) in zip(grids, scs, alone):
        assert g.step_count == steps
        for c in range(6):
            assert np.array_equal(g.get_field(c), fa[c])
        for p in range(len(sc.probes)):
            assert np.array_equal(g.read_probe(p), pa[p])
    b.close()
    for g in grids:
        g.close()


def test_batch_grounding_domains_vs_oracle(fdtd):
    """three grounding-rod domains of the batched workload (48..56 cells,
    8-cell CPML, random soil, rod, riser and leads), 300 steps from rest:
    gap voltage and source current within 1e-4 of the FP64 oracle"""
    rng = np.random.default_rng(7)
    scs = []
    for n in (48, 52, 56):
        scs.append(W.grounding_domain(n, rng.uniform(4, 40), 10 ** rng.uniform(-4, -1),
                                      rng.uniform(1.0, 0.25 * (n - 28)), 0.008, 0.0, 0.25e-6, n_steps=300))
    grids = [fdtd.from_scenario(sc, probe_capacity=300) for sc in scs]
    b = fdtd.Batch(grids)
    b.step(300)
    b.synchronize()
    for g, sc in zip(grids, scs):
        o = oracle_from_scenario(sc, parity=True)
        o.step(300)
        for p in range(len(sc.probes)):
            assert rel_l2(g.read_probe(p), o.read_probe(p)) <= 1e-4
    b.close()
    for g in grids:
        g.close()


def test_batch_inclined_grounding_domains_vs_oracle(fdtd):
    """three domains of the inclined-rod batched workload (rods of 1.5..4 m
    leaning 20..60 degrees: oblique wires joined to the risers), 300 steps
    from rest in one batch: gap voltage, source current, the rod's segment
    currents and node charges within 1e-4 of the FP64 oracle"""
    import math
    rng = np.random.default_rng(8)
    scs = []
    for n, deg in ((48, 20), (52, 45), (56, 60)):
        scs.append(W.grounding_domain(n, rng.uniform(4, 40), 10 ** rng.uniform(-4, -1), rng.uniform(1.5, 4.0),
                                      0.008, 0.0, 0.25e-6, n_steps=300, incline=math.radians(deg),
                                      courant=W.INCLINED_COURANT))
    grids = [fdtd.from_scenario(sc, probe_capacity=300) for sc in scs]
    b = fdtd.Batch(grids)
    b.step(300)
    b.synchronize()
    for g, sc in zip(grids, scs):
        o = oracle_from_scenario(sc, parity=True)
        o.step(300)
        for p in range(len(sc.probes)):
            assert rel_l2(g.read_probe(p), o.read_probe(p)) <= 1e-4
        I, Q = g.get_wire_state()
        Io, Qo = o.get_wire_state()
        assert rel_l2(I, Io) <= 1e-4 and rel_l2(Q, Qo) <= 1e-4
        assert float(np.abs(Io).max()) > 100.0                 # the rod carries the feed current
    b.close()
    for g in grids:
        g.close()


def test_batch_rejects_mismatched_steps(fdtd):
    a = build(fdtd, W.random_scenario(1, n=(10, 10, 10), n_steps=4), 4)
    c = build(fdtd, W.random_scenario(2, n=(12, 10, 9), n_steps=4), 4)
    a.step(1)
    with pytest.raises(fdtd.FdtdError):
        fdtd.Batch([a, c])
    a.close()
    c.close()


def test_config4_full_batch_sampled_domains(fdtd):
    """The whole batched workload (256 grounding domains, sides 48..128,
    8-cell CPML) in the launch shape the benchmark times (tuned tile depth
    per size class): four sampled domains (smallest, largest, two seeded
    picks) start from random fields, the rest from rest; after 40 steps
    every field of the sampled domains is within 1e-5 of the FP64 oracle and
    their probes within 1e-4."""
    from paper_2207_06908_gb300 import grounding
    steps = 40
    scs = W.config4(n_steps=steps)
    sizes = [sc.n[0] for sc in scs]
    rng = np.random.default_rng(44)
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    while len(picks) < 4:
        picks.add(int(rng.integers(0, len(scs))))
    for q in picks:
        scs[q].fields = W.random_fields(np.random.default_rng(1000 + q), scs[q].n)
    blocks = {}
    for sc in scs:
        c = grounding.size_class(sc.n[0])
        if c not in blocks:
            blocks[c] = grounding.tune_block(sc.n[0])
    grids = [fdtd.from_scenario(sc, probe_capacity=steps, block=blocks[grounding.size_class(sc.n[0])])
             for sc in scs]
    for q in picks:
        for c, f in enumerate(scs[q].fields):
            grids[q].set_field(c, f)
    b = fdtd.Batch(grids)
    b.step(steps)
    b.synchronize()
    for q in sorted(picks):
        sc, g = scs[q], grids[q]
        o = oracle_from_scenario(sc, parity=True)
        o.step(steps)
        for c in range(6):
            assert rel_l2(g.get_field(c), o.get_field(c)) <= 1e-5, (q, sc.n, c)
        for p in range(len(sc.probes)):
            ref = o.read_probe(p)
            if np.linalg.norm(ref) > 0:
                assert rel_l2(g.read_probe(p), ref) <= 1e-4, (q, p)
    b.close()
    for g in grids:
        g.close()


def test_one_domain_batch_between_single_steps(fdtd):
    """a grid stepped 3 times alone (odd parity), then as a one-domain batch
    for 30 steps (direct launches until the parity allows a graph), then 5
    more times alone, equals the same grid stepped 38 times alone, bit for
    bit (fields and every probe sample)"""
    sc = W.random_scenario(321, n=(37, 29, 23), cpml=4, n_steps=38)
    ref = build(fdtd, sc, 38)
    ref.step(38)
    want = [ref.get_field(c) for c in range(6)], [ref.read_probe(p) for p in range(len(sc.probes))]
    ref.close()
    g = build(fdtd, sc, 38)
    g.step(3)
    b = fdtd.Batch([g])
    b.step(30)
    b.synchronize()
    b.close()
    g.step(5)
    assert g.step_count == 38
    for c in range(6):
        assert np.array_equal(g.get_field(c), want[0][c])
    for p in range(len(sc.probes)):
        assert np.array_equal(g.read_probe(p), want[1][p])
    g.close()
