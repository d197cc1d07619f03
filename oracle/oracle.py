"""Python handle on the FP64 CPU FDTD oracle (fdtd_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of ``bench.py`` are the only callers.  The CUDA
library never imports this module and this module never imports the
library.

The C file follows the paper's Sec. 2.1 (Eq. maxwell, maxwelle, maxwellh,
fdtdex, fdtdhx), Sec. 2.2 (CPML), Sec. 2.3 (thin wires, axis-aligned and
oblique) and the "calculate" probes of the Sec. 4 model files; see its
header for the readings taken.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc_fdtd.so")
_SO32 = os.path.join(_BUILD, "liborc_fdtd_f32.so")
_lock = threading.Lock()
_libs = {}

PROBE_V, PROBE_I, PROBE_E, PROBE_H = 0, 1, 2, 3
EX, EY, EZ, HX, HY, HZ = range(6)

C0 = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6


def _build_one(so: str, defs: list[str], force: bool) -> str:
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(_SRC)):
        return so
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", *defs,
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction): the FP64
    oracle, and the same source with FP32 storage and arithmetic, which
    only serves to size the rounding error of FP32 field storage."""
    os.makedirs(_BUILD, exist_ok=True)
    _build_one(_SO32, ["-DORC_REAL=float"], force)
    return _build_one(_SO, [], force)


def _load(f32: bool = False):
    with _lock:
        if f32 in _libs:
            return _libs[f32]
        build()
        lib = ctypes.CDLL(_SO32 if f32 else _SO)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [I, I, I, D, D, I]
        lib.orc_destroy.argtypes = [P]
        lib.orc_dt.restype = D
        lib.orc_dt.argtypes = [P]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_step_count.restype = ctypes.c_long
        lib.orc_step_count.argtypes = [P]
        lib.orc_set_cpml.argtypes = [P, I, D, D, D, D, D]
        lib.orc_set_materials.argtypes = [P, u8p, dp, dp, dp, I]
        lib.orc_add_wire.argtypes = [P, I, I, I, I, I, I, D]
        lib.orc_add_source.argtypes = [P, I, I, I, I, dp, I]
        lib.orc_add_probe.argtypes = [P, I, I, I, I, I, I]
        lib.orc_finalize.argtypes = [P, I]
        lib.orc_set_field.argtypes = [P, I, dp]
        lib.orc_get_field.argtypes = [P, I, dp]
        lib.orc_get_coef.argtypes = [P, I, dp]
        lib.orc_step.argtypes = [P, I]
        lib.orc_read_probe.argtypes = [P, I, dp]
        lib.orc_set_debye.argtypes = [P, I, I, dp, dp]
        lib.orc_add_source_r.argtypes = [P, I, I, I, I, D, dp, I]
        lib.orc_add_vsource.argtypes = [P, I, I, I, I, D, dp, I]
        lib.orc_add_lumped.argtypes = [P, I, I, I, I, D, D]
        lib.orc_add_wire_path.argtypes = [P, I, I, I, I, I, I, D]
        lib.orc_get_debye_current.argtypes = [P, I, I, dp]
        lib.orc_set_debye_current.argtypes = [P, I, I, dp]
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_add_owire.argtypes = [P, D, D, D, D, D, D, D]
        lib.orc_add_owire_vsource.argtypes = [P, I, I, D, dp, I]
        lib.orc_add_owire_probe.argtypes = [P, I, I]
        lib.orc_add_owire_node_probe.argtypes = [P, D, D, D]
        lib.orc_owire_counts.argtypes = [P, ip, ip]
        lib.orc_owire_counts.restype = None
        lib.orc_get_owire_state.argtypes = [P, dp, dp]
        lib.orc_set_owire_state.argtypes = [P, dp, dp]
        lib.orc_get_owire_coefs.argtypes = [P, dp, dp]
        _libs[f32] = lib
        return lib


def num_threads() -> int:
    """OpenMP threads the oracle's update loops run on."""
    return _load().orc_num_threads()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


class OracleGrid:
    """One FP64 simulation domain.

    Arrays are exchanged in the cell-owned layout: shape (nz, ny, nx), entry
    [k, j, i] = Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2), Hx(i,j+1/2,k+1/2),
    Hy(i+1/2,j,k+1/2) or Hz(i+1/2,j+1/2,k).
    """

    def __init__(self, nx, ny, nz, dx, courant=0.99, parity=False, f32=False):
        """parity: round coefficients and source samples to FP32 (arithmetic
        stays FP64).  f32: the FP32-storage build of the same algorithm (a
        yardstick for FP32 rounding, not a reference)."""
        self._lib = _load(f32)
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dx = dx
        h = self._lib.orc_create(nx, ny, nz, float(dx), float(courant), int(bool(parity)))
        if not h:
            raise ValueError("oracle rejected the grid")
        self._h = h
        self.n_probes = 0
        self.max_steps = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def dt(self) -> float:
        return self._lib.orc_dt(self._h)

    @property
    def step_count(self) -> int:
        return self._lib.orc_step_count(self._h)

    def set_cpml(self, cells, order=3.0, kappa_max=1.0, alpha_max=0.0, alpha_order=1.0,
                 sigma_max=0.0):
        _check(self._lib.orc_set_cpml(self._h, int(cells), order, kappa_max, alpha_max,
                                      alpha_order, sigma_max), "set_cpml")

    def set_materials(self, cell_material, eps_r, sigma, mu_r):
        cm = np.ascontiguousarray(cell_material, dtype=np.uint8)
        assert cm.shape == self.shape
        e = np.ascontiguousarray(eps_r, dtype=np.float64)
        s = np.ascontiguousarray(sigma, dtype=np.float64)
        m = np.ascontiguousarray(mu_r, dtype=np.float64)
        _check(self._lib.orc_set_materials(
            self._h, cm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
            _dptr(e), _dptr(s), _dptr(m), len(e)), "set_materials")

    def add_wire_path(self, p0, p1, radius):
        """wire between two arbitrary nodes as a staircase of grid-aligned
        segments; returns the number of segments"""
        rc = self._lib.orc_add_wire_path(self._h, *map(int, p0), *map(int, p1), float(radius))
        if rc < 0:
            raise ValueError(f"oracle add_wire_path failed with status {rc}")
        return rc

    def set_debye(self, material, deps, tau):
        """Debye poles (relative delta eps, tau in s) of one material"""
        d = np.ascontiguousarray(deps, dtype=np.float64)
        t = np.ascontiguousarray(tau, dtype=np.float64)
        _check(self._lib.orc_set_debye(self._h, int(material), len(d), _dptr(d), _dptr(t)), "set_debye")

    def set_debye_current(self, comp, pole, values):
        """J_p at the current E time level t_n of E component comp
        (cell-owned layout)"""
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.shape == self.shape
        _check(self._lib.orc_set_debye_current(self._h, int(comp), int(pole), _dptr(v)), "set_debye_current")

    def get_debye_current(self, comp, pole) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        _check(self._lib.orc_get_debye_current(self._h, int(comp), int(pole), _dptr(out)), "get_debye_current")
        return out

    def add_wire(self, p0, p1, radius):
        _check(self._lib.orc_add_wire(self._h, *map(int, p0), *map(int, p1), float(radius)),
               "add_wire")

    def add_source(self, node, axis, current, r_internal=0.0):
        """current source (A at t_{n+1/2}); r_internal > 0: in parallel"""
        cur = np.ascontiguousarray(current, dtype=np.float64)
        _check(self._lib.orc_add_source_r(self._h, *map(int, node), int(axis), float(r_internal), _dptr(cur),
                                          len(cur)), "add_source")

    def add_voltage_source(self, node, axis, voltage, r_internal=0.0):
        """voltage source V = -E dx across the edge: ideal (r_internal = 0,
        V at t_{n+1}) or with a series resistance (V at t_{n+1/2})"""
        v = np.ascontiguousarray(voltage, dtype=np.float64)
        _check(self._lib.orc_add_vsource(self._h, *map(int, node), int(axis), float(r_internal), _dptr(v),
                                         len(v)), "add_voltage_source")

    def add_lumped(self, node, axis, resistance=0.0, capacitance=0.0):
        _check(self._lib.orc_add_lumped(self._h, *map(int, node), int(axis), float(resistance),
                                        float(capacitance)), "add_lumped")

    def add_oblique_wire(self, p0, p1, radius):
        """straight wire between two points in node units (any
        orientation, floats allowed); returns its index"""
        rc = self._lib.orc_add_owire(self._h, *map(float, p0), *map(float, p1), float(radius))
        if rc < 0:
            _check(rc, "add_oblique_wire")
        return rc

    def add_wire_voltage_source(self, wire, segment, voltage, r_internal=0.0):
        """delta-gap EMF (V at t_n) with series resistance r_internal in one
        segment of an oblique wire, driving current from the segment's start
        towards its end"""
        v = np.ascontiguousarray(voltage, dtype=np.float64)
        _check(self._lib.orc_add_owire_vsource(self._h, int(wire), int(segment), float(r_internal), _dptr(v),
                                               len(v)), "add_wire_voltage_source")

    def add_wire_probe(self, wire, segment):
        """current of one segment of an oblique wire at t_{n+1/2}"""
        _check(self._lib.orc_add_owire_probe(self._h, int(wire), int(segment)), "add_wire_probe")
        self.n_probes += 1
        return self.n_probes - 1

    def add_wire_node_probe(self, point):
        """in-cell potential of the oblique-wire node at point, at t_{n+1}"""
        _check(self._lib.orc_add_owire_node_probe(self._h, *map(float, point)), "add_wire_node_probe")
        self.n_probes += 1
        return self.n_probes - 1

    def wire_counts(self):
        ns, nn = ctypes.c_int(), ctypes.c_int()
        self._lib.orc_owire_counts(self._h, ctypes.byref(ns), ctypes.byref(nn))
        return ns.value, nn.value

    def get_wire_state(self):
        """(I_s at the last half step, Q_m at the current step)"""
        ns, nn = self.wire_counts()
        I, Q = np.zeros(max(ns, 1)), np.zeros(max(nn, 1))
        _check(self._lib.orc_get_owire_state(self._h, _dptr(I), _dptr(Q)), "get_wire_state")
        return I[:ns], Q[:nn]

    def set_wire_state(self, I, Q):
        I = np.ascontiguousarray(I, dtype=np.float64)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        _check(self._lib.orc_set_owire_state(self._h, _dptr(I), _dptr(Q)), "set_wire_state")

    def get_wire_coefs(self):
        """per segment L' dl (H), per node 1 / (C' dl_m) (0 when grounded)"""
        ns, nn = self.wire_counts()
        L, cV = np.zeros(max(ns, 1)), np.zeros(max(nn, 1))
        _check(self._lib.orc_get_owire_coefs(self._h, _dptr(L), _dptr(cV)), "get_wire_coefs")
        return L[:ns], cV[:nn]

    def add_probe(self, kind, node, axis, n_edges=1):
        _check(self._lib.orc_add_probe(self._h, int(kind), *map(int, node), int(axis),
                                       int(n_edges)), "add_probe")
        self.n_probes += 1
        return self.n_probes - 1

    def finalize(self, max_steps=0):
        _check(self._lib.orc_finalize(self._h, int(max_steps)), "finalize")
        self.max_steps = int(max_steps)

    def set_field(self, comp, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.shape == self.shape
        _check(self._lib.orc_set_field(self._h, int(comp), _dptr(v)), "set_field")

    def get_field(self, comp) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        _check(self._lib.orc_get_field(self._h, int(comp), _dptr(out)), "get_field")
        return out

    def get_coef(self, which) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        _check(self._lib.orc_get_coef(self._h, int(which), _dptr(out)), "get_coef")
        return out

    def step(self, n):
        _check(self._lib.orc_step(self._h, int(n)), "step")

    @classmethod
    def from_scenario(cls, sc, parity=True, f32=False):
        """Build from a problem description with the attributes n, dx,
        courant, cpml, cell_material, materials [(eps_r, sigma, mu_r)],
        wires [(p0, p1, radius)], sources [(node, axis, current)], probes
        [(kind, node, axis, n_edges)], n_steps, fields (or None) and debye
        {material: (deps, tau)} (optional)."""
        g = cls(*sc.n, sc.dx, courant=sc.courant, parity=parity, f32=f32)
        if sc.cpml:
            g.set_cpml(sc.cpml)
        g.set_materials(sc.cell_material, [m[0] for m in sc.materials], [m[1] for m in sc.materials],
                        [m[2] for m in sc.materials])
        for mat, (deps, tau) in (getattr(sc, "debye", None) or {}).items():
            g.set_debye(mat, deps, tau)
        for p0, p1, r in sc.wires:
            g.add_wire(p0, p1, r)
        for p0, p1, r in getattr(sc, "wire_paths", None) or []:
            g.add_wire_path(p0, p1, r)
        for src in sc.sources:
            node, axis, cur = src[:3]
            g.add_source(node, axis, cur, *(src[3:4]))
        for node, axis, volt, r in getattr(sc, "vsources", None) or []:
            g.add_voltage_source(node, axis, volt, r)
        for node, axis, res, cap in getattr(sc, "lumped", None) or []:
            g.add_lumped(node, axis, res, cap)
        for p0, p1, r in getattr(sc, "owires", None) or []:
            g.add_oblique_wire(p0, p1, r)
        for src in getattr(sc, "owire_sources", None) or []:
            g.add_wire_voltage_source(*src)
        for kind, node, axis, ne in sc.probes:
            g.add_probe(kind, node, axis, ne)
        for pr in getattr(sc, "owire_probes", None) or []:
            if len(pr) == 3:
                g.add_wire_node_probe(pr)
            else:
                g.add_wire_probe(*pr)
        g.finalize(sc.n_steps)
        if sc.fields is not None:
            # start from the FP32-rounded fields the GPU starts from
            for c, f in enumerate(sc.fields):
                g.set_field(c, np.asarray(f, dtype=np.float32).astype(np.float64))
        return g

    def read_probe(self, p) -> np.ndarray:
        out = np.empty(max(self.max_steps, 1), dtype=np.float64)
        _check(self._lib.orc_read_probe(self._h, int(p), _dptr(out)), "read_probe")
        return out[: self.max_steps]
