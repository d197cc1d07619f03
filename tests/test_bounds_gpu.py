"""The bounds-checked build: the library compiled with -DFDTD_BOUNDS tests
every global access of its step and source/probe kernels against the
array's extent.  Run on scenarios that exercise every path (PEC and CPML
grids with ragged sizes, thin and oblique wires, sources and probes of
every kind, Debye media, a batch), it must record no access outside an
array, and give the release build's results."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2207_06908_gb300 import _lib, fdtd, workloads as W
out = {"reports": [], "sums": []}
import ctypes
def report(g):
    s, c = ctypes.c_int(), ctypes.c_int()
    rc = g._lib.fdtd_bounds_report(g._h, ctypes.byref(s), ctypes.byref(c))
    out["reports"].append([rc, s.value, c.value])
def run(sc, steps):
    g = fdtd.from_scenario(sc, probe_capacity=steps)
    if sc.fields is not None:
        for c, f in enumerate(sc.fields):
            g.set_field(c, f)
    g.step(steps)
    out["sums"].append(float(sum(np.abs(g.get_field(c)).astype(np.float64).sum() for c in range(6))))
    n = len(sc.probes) + len(getattr(sc, "owire_probes", None) or [])
    out["sums"].append(float(sum(np.abs(g.read_probe(p)).astype(np.float64).sum() for p in range(n))))
    report(g)
    g.close()
run(W.random_scenario(3, n=(17, 17, 17), n_steps=40), 40)
run(W.random_scenario(104, n=(45, 21, 27), cpml=5, n_steps=40), 40)
sc = W.random_scenario(43, n=(24, 20, 18), cpml=3, n_wires=0, n_steps=40, courant=0.9)
sc = W.with_random_debye(sc, 5, materials=(0, 1, 2, 3), max_poles=2)
J = (11.5, 9.25, 8.75)
sc.owires = [((5.0, 5.5, 5.0), J, 0.004), (J, (18.5, 14.0, 12.5), 0.002)]
sc.owire_probes = [(1, 2), J]
run(sc, 40)
scs = [W.random_scenario(200 + q, n=n, cpml=c, n_steps=35) for q, (n, c) in enumerate([((17, 17, 17), 0), ((45, 21, 27), 5), ((33, 40, 18), 3)])]
gs = [fdtd.from_scenario(s, probe_capacity=35) for s in scs]
for g, s in zip(gs, scs):
    for c, f in enumerate(s.fields):
        g.set_field(c, f)
b = fdtd.Batch(gs)
b.step(35)
b.synchronize()
for g in gs:
    out["sums"].append(float(sum(np.abs(g.get_field(c)).astype(np.float64).sum() for c in range(6))))
    report(g)
b.close()
for g in gs:
    g.close()
print(json.dumps(out))
'''


def run_child(env):
    code = "ROOT = %r\n" % ROOT + CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_records_no_stray_access():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import _build
    lib = _build.build_bounds()
    checked = run_child(dict(os.environ, FDTD_LIBRARY=lib))
    release = run_child({k: v for k, v in os.environ.items() if k != "FDTD_LIBRARY"})
    for rc, site, count in checked["reports"]:
        assert rc == 0 and count == 0, (site, count)
    assert all(rc == 1 for rc, _, _ in release["reports"])       # the release build checks nothing
    np.testing.assert_allclose(checked["sums"], release["sums"], rtol=1e-6)
