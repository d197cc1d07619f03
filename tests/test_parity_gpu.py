"""GPU (FP32, through the C ABI) against the FP64 oracle in parity mode
(coefficients and source samples rounded to FP32, arithmetic in FP64).

Tolerances: relative L2 <= 1e-5 on every field component and <= 1e-4 on
every probe waveform, on the same seeded inputs.
"""
import os

import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W
from _scenario import COMPONENTS, field_errors, oracle_from_scenario, record, rel_l2

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FIELD_TOL = 1e-5
PROBE_TOL = 1e-4


@pytest.fixture(scope="module")
def fdtd():
    import torch
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
    fields = [g.get_field(c) for c in range(6)]
    probes = [g.read_probe(p, 0, steps) for p in range(len(sc.probes))]
    g.close()
    return fields, probes


def run_oracle(sc, steps):
    o = oracle_from_scenario(sc, parity=True)
    o.step(steps)
    return [o.get_field(c) for c in range(6)], [o.read_probe(p)[:steps] for p in range(len(sc.probes))]


def compare(gf, gp, of, op, field_tol=FIELD_TOL, probe_tol=PROBE_TOL, steps=None):
    errs = []
    for c, (e, norm) in enumerate(field_errors(gf, of)):
        errs.append(e)
        record(None, f"field {COMPONENTS[c]}", e, field_tol, steps=steps, norm=norm)
    for p in range(len(gp)):
        if np.linalg.norm(op[p]) == 0:
            assert np.all(gp[p] == 0)
            continue
        e = rel_l2(gp[p], op[p])
        record(None, f"probe {p}", e, probe_tol, steps=steps)
        assert e <= probe_tol, f"probe {p}: rel L2 {e:.3e}"
    for c, e in enumerate(errs):
        assert e <= field_tol, f"component {c}: rel L2 {e:.3e}"
    return errs


@pytest.mark.parametrize("seed", range(6))
def test_random_pec_17cube(fdtd, seed):
    """random blocky media, wires, sources, probes and fields; 17^3 spans
    one full 32x8 tile row plus a ragged tail in y and two z chunks"""
    sc = W.random_scenario(seed, n=(17, 17, 17), n_steps=60)
    compare(*run_gpu(fdtd, sc, 60), *run_oracle(sc, 60))


@pytest.mark.parametrize("seed", range(4))
def test_random_cpml_ragged(fdtd, seed):
    """odd, non-multiple-of-tile sizes with a CPML on all faces"""
    sc = W.random_scenario(100 + seed, n=(45, 21, 27), cpml=5, n_steps=70)
    compare(*run_gpu(fdtd, sc, 70), *run_oracle(sc, 70))


def test_smallest_grid(fdtd):
    """degenerate 2x2x2 box: every E is a wall except none; H only"""
    sc = W.random_scenario(7, n=(2, 3, 2), n_wires=0, n_sources=0, n_probes=0, n_steps=5)
    compare(*run_gpu(fdtd, sc, 5), *run_oracle(sc, 5))


def test_zero_steps_leaves_fields(fdtd):
    sc = W.random_scenario(8, n=(9, 10, 11), n_steps=4)
    g = fdtd.from_scenario(sc, probe_capacity=4)
    for c, f in enumerate(sc.fields):
        g.set_field(c, f)
    g.step(0)
    for c, f in enumerate(sc.fields):
        assert np.array_equal(g.get_field(c), np.asarray(f, np.float32))
    g.close()


def test_random_long_500(fdtd):
    """500 steps from random fields over random media, wires and weak
    sources (CPML on): fields stay within 1e-5 of the FP64 oracle"""
    sc = W.random_scenario(31, n=(36, 29, 26), cpml=4, n_steps=500, current_scale=1e-3)
    compare(*run_gpu(fdtd, sc, 500), *run_oracle(sc, 500))


def compare_from_rest(sc, n, gf, gp, of, op):
    """fields: max(1e-5, 2x the FP32-storage error of the same algorithm);
    probes: max(1e-4, 2x that error of the probe).  Every error achieved is
    recorded beside both bars."""
    from oracle.oracle import OracleGrid
    y = OracleGrid.from_scenario(sc, parity=True, f32=True)
    y.step(n)
    yp = [y.read_probe(p)[:n] for p in range(len(gp))]
    fails = []
    yards = field_errors([y.get_field(c) for c in range(6)], of)
    for c, ((e, norm), (yard, _)) in enumerate(zip(field_errors(gf, of), yards)):
        bar = max(FIELD_TOL, 2.0 * yard)
        record(None, f"field {COMPONENTS[c]}", e, bar, fp32_yardstick=yard, steps=n, norm=norm)
        if not e <= bar:
            fails.append(f"component {c}: rel L2 {e:.3e} > {bar:.3e}")
    del y
    for p in range(len(gp)):
        e = rel_l2(gp[p], op[p])
        yard = rel_l2(yp[p], op[p])
        bar = max(PROBE_TOL, 2.0 * yard)
        record(None, f"probe {p}", e, bar, fp32_yardstick=yard, steps=n)
        if not e <= bar:
            fails.append(f"probe {p}: rel L2 {e:.3e} > {bar:.3e}")
    assert not fails, "; ".join(fails)


def test_config1_full(fdtd):
    """48^3 PEC lossy half-space, Gaussian-derivative source, 500 steps from
    rest.  Probes: 1e-4.  Fields: the 1 A source drives a near field of
    ~2e4 V/m while the field left at step 500 has an rms of ~0.1 V/m, so
    rounding any FP32 store of the near field costs more than 1e-5 of the
    final field; the bar is max(1e-5, 2x the error of the same algorithm
    evaluated with FP32 storage on the CPU)."""
    sc = W.config1()
    n = sc.n_steps
    compare_from_rest(sc, n, *run_gpu(fdtd, sc, n), *run_oracle(sc, n))


def test_graph_and_direct_paths_agree(fdtd):
    """fdtd_step replays a captured graph of 32 steps plus direct launches;
    any split of the same step count gives bitwise the same state"""
    sc = W.random_scenario(21, n=(40, 18, 33), cpml=4, n_steps=75)
    a_f, a_p = run_gpu(fdtd, sc, 75)
    g = fdtd.from_scenario(sc, probe_capacity=75)
    for c, f in enumerate(sc.fields):
        g.set_field(c, f)
    for n in (1, 2, 33, 7, 32):
        g.step(n)
    b_f = [g.get_field(c) for c in range(6)]
    b_p = [g.read_probe(p, 0, 75) for p in range(len(sc.probes))]
    g.close()
    for x, y in zip(a_f, b_f):
        assert np.array_equal(x, y)
    for x, y in zip(a_p, b_p):
        assert np.array_equal(x, y)


def test_config2_full_size_truncated(fdtd):
    """256^3, 10-cell CPML, thin wire, source and probes: the bench workload
    at full size, in the bench's launch path (one 32-step graph + direct
    steps), from seeded random fields so every cell is active; 40 steps.
    The 10 kA source's near field dwarfs the 1 V/m random fields, so the
    field bar is the one of the from-rest runs."""
    steps = 40
    sc = W.config2(n_steps=steps)
    rng = np.random.default_rng(2024)
    sc.fields = W.random_fields(rng, sc.n)
    compare_from_rest(sc, steps, *run_gpu(fdtd, sc, steps), *run_oracle(sc, steps))


def test_config2_full_size_random_fields_no_source(fdtd):
    """the same 256^3 grid (CPML, wire classes, probes) without the source:
    every cell active, fields within 1e-5 after 40 steps"""
    steps = 40
    sc = W.config2(n_steps=steps)
    sc.sources = []
    rng = np.random.default_rng(2025)
    sc.fields = W.random_fields(rng, sc.n)
    compare(*run_gpu(fdtd, sc, steps), *run_oracle(sc, steps))


def test_config3_full_size_random_fields_no_source(fdtd):
    """512x512x384, 12-cell CPML, two-layer soil, the buried 8x8 wire mesh,
    down-conductor and leads (the largest workload, 100.7 M cells) at full
    size without its source, from seeded random fields: fields within 1e-5
    and probes within 1e-4 after 12 steps"""
    steps = 12
    sc = W.config3(n_steps=steps)
    sc.sources = []
    rng = np.random.default_rng(2026)
    sc.fields = W.random_fields(rng, sc.n)
    compare(*run_gpu(fdtd, sc, steps), *run_oracle(sc, steps))


def test_config2_scaled_long_run(fdtd):
    """the config-2 layout at 64^3 for 800 steps from rest: the source
    drives the wire through the CPML window (from rest: the field bar of
    test_config1_full)"""
    sc = W.config2(n_steps=800, n=64)
    compare_from_rest(sc, 800, *run_gpu(fdtd, sc, 800), *run_oracle(sc, 800))


def test_wide_index_instantiation_is_bitwise_equal():
    """grids of 2^31 elements or more step with 64-bit field indices (another
    instantiation of the step kernel); forced on a small CPML grid in a
    child process (FDTD_WIDE_INDEX=1), it gives bit for bit the fields and
    probes of the 32-bit instantiation"""
    import subprocess
    import sys
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    code = (
        "import sys, numpy as np; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "from paper_2207_06908_gb300 import fdtd as F, workloads as W\n"
        "sc = W.random_scenario(52, n=(45, 21, 27), cpml=5, n_steps=70)\n"
        "g = F.from_scenario(sc, probe_capacity=70)\n"
        "[g.set_field(c, f) for c, f in enumerate(sc.fields)]\n"
        "g.step(70)\n"
        "np.savez(sys.argv[1], *[g.get_field(c) for c in range(6)], *[g.read_probe(p) for p in range(len(sc.probes))])\n"
    ) % (ROOT, os.path.join(ROOT, "tests"))
    outs = []
    for wide in ("0", "1"):
        path = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"fdtd_wide_{os.getpid()}_{wide}.npz")
        env = dict(os.environ, FDTD_WIDE_INDEX=wide)
        subprocess.run([sys.executable, "-c", code, path], check=True, env=env)
        z = np.load(path)
        outs.append([z[k] for k in z.files])
        os.remove(path)
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
