"""Checkpoint / resume through the C ABI (GPU): a grid that loads a saved
state continues bit for bit as the grid that saved it."""
import numpy as np
import pytest

from paper_2207_06908_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdtd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import fdtd as F
    return F


def state_of(g, sc):
    return [g.get_field(c) for c in range(6)], [g.read_probe(p) for p in range(len(sc.probes))]


@pytest.mark.parametrize("cpml,first", [(4, 21), (0, 32)])
def test_resume_is_bitwise(fdtd, cpml, first):
    """save after `first` steps (odd: the loading grid's buffer parity
    differs), run 45 more on the saver and, after loading, on a fresh grid
    built from the same description; also rewind the saver itself"""
    total = first + 45
    sc = W.random_scenario(31 + cpml, n=(40, 18, 33), cpml=cpml, n_steps=total)
    a = fdtd.from_scenario(sc, probe_capacity=total)
    for c, f in enumerate(sc.fields):
        a.set_field(c, f)
    a.step(first)
    st = a.save_state()
    a.step(total - first)
    fa, pa = state_of(a, sc)
    b = fdtd.from_scenario(sc, probe_capacity=total)
    b.load_state(st)
    assert b.step_count == first
    b.step(total - first)
    fb, pb = state_of(b, sc)
    a.load_state(st)
    a.step(total - first)
    fa2, pa2 = state_of(a, sc)
    for x, y, z in zip(fa, fb, fa2):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    for x, y, z in zip(pa, pb, pa2):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    assert np.abs(fa[2]).max() > 0
    a.close()
    b.close()


def test_load_rejects_other_shapes(fdtd):
    sc = W.random_scenario(5, n=(20, 13, 18), cpml=3, n_steps=10)
    g = fdtd.from_scenario(sc, probe_capacity=10)
    g.step(4)
    st = g.save_state()
    other = W.random_scenario(5, n=(20, 13, 19), cpml=3, n_steps=10)
    h = fdtd.from_scenario(other, probe_capacity=10)
    with pytest.raises(fdtd.FdtdError):
        h.load_state(st)
    with pytest.raises(fdtd.FdtdError):
        g.load_state(st[: len(st) // 2])
    with pytest.raises(fdtd.FdtdError):
        g.load_state(b"\0" * len(st))
    g.close()
    h.close()
