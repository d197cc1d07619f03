"""Edge cases of the GPU path against the FP64 oracle: coefficient classes
near the 256 limit, the thinnest grid a CPML allows, extreme aspect ratios,
probes beyond their capacity."""
import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W
from _scenario import oracle_from_scenario, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd as F
    return F


def run_both(F, sc, steps, capacity=None):
    g = F.from_scenario(sc, probe_capacity=steps if capacity is None else capacity)
    for c, f in enumerate(sc.fields):
        g.set_field(c, f)
    g.step(steps)
    gf = [g.get_field(c) for c in range(6)]
    ncls = g.num_classes
    o = oracle_from_scenario(sc, parity=True)
    o.step(steps)
    of = [o.get_field(c) for c in range(6)]
    for c in range(6):
        assert rel_l2(gf[c], of[c]) <= 1e-5, c
    return g, o, ncls


def layered(n, n_layers, seed, cpml=0):
    """one material per z plane group: distinct coefficient sets at every
    layer and every interface"""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    cm = np.zeros((nz, ny, nx), np.uint8)
    for k in range(nz):
        cm[k] = k * n_layers // nz
    mats = [(float(rng.uniform(1, 30)), float(10 ** rng.uniform(-4, -1)), float(rng.uniform(1, 3)))
            for _ in range(n_layers)]
    sc = W.Scenario("layered", n, 0.1, 0.99, cpml, cm, mats, n_steps=40)
    sc.fields = W.random_fields(rng, n)
    return sc


def test_classes_near_the_limit(fdtd):
    """32 layers of random media over 200 planes fill the coefficient table
    close to its 256 entries (each interface adds the mixed sets of the
    edges that straddle it); one more layer overflows it"""
    sc = layered((18, 17, 200), 32, 3)
    g, _, ncls = run_both(fdtd, sc, 40)
    assert 200 <= ncls <= 256, ncls
    g.close()
    with pytest.raises(fdtd.FdtdError, match="ECLASSES"):
        fdtd.from_scenario(layered((18, 17, 200), 33, 3), probe_capacity=1)


@pytest.mark.parametrize("d", [3, 6])
def test_thinnest_cpml_grid(fdtd, d):
    """every axis 2d + 2 cells (the least a CPML of d cells allows): every
    tile meets both layers of x and y, every plane is in a z layer or next
    to one"""
    n = (2 * d + 2,) * 3
    sc = W.random_scenario(70 + d, n=n, cpml=d, n_wires=0, n_sources=0, n_probes=4, n_steps=30)
    g, _, _ = run_both(fdtd, sc, 30)
    g.close()


@pytest.mark.parametrize("n", [(200, 3, 3), (3, 150, 4), (5, 4, 180), (67, 2, 41)])
def test_extreme_aspect_ratios(fdtd, n):
    sc = W.random_scenario(sum(n), n=n, n_wires=0, n_sources=0, n_probes=0, n_steps=25)
    g, _, _ = run_both(fdtd, sc, 25)
    g.close()


def test_probes_beyond_capacity(fdtd):
    """a run longer than the probe capacity records the first samples only
    and reading past the capacity is an error"""
    sc = W.random_scenario(81, n=(15, 14, 13), n_steps=30)
    g, o, _ = run_both(fdtd, sc, 30, capacity=12)
    for p in range(len(sc.probes)):
        got = g.read_probe(p, 0, 12)
        ref = o.read_probe(p)[:12]
        if np.linalg.norm(ref) > 0:
            assert rel_l2(got, ref) <= 1e-4
    with pytest.raises(fdtd.FdtdError):
        g.read_probe(0, 10, 5)
    g.close()
