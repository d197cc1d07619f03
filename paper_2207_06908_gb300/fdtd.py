"""Python face of the C ABI (include/fdtd.h): one ``Grid`` per simulation
domain.  Argument marshalling only -- every update runs in the CUDA library.

PyTorch supplies the CUDA stream and, by default, the device memory (one
uint8 tensor that the library carves into fields, classes, CPML state,
sources and probe buffers).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import CpmlParams, FdtdError, Material, check

EX, EY, EZ, HX, HY, HZ = range(6)
PROBE_V, PROBE_I, PROBE_E, PROBE_H, PROBE_WIRE, PROBE_WIRE_V = 0, 1, 2, 3, 4, 5


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Grid:
    """A uniform cubic Yee grid of nx*ny*nz cells (Sec. 2.1 of the paper).

    Host arrays use the cell-owned layout of shape (nz, ny, nx): entry
    [k, j, i] is the component owned by cell (i, j, k).
    """

    def __init__(self, nx, ny, nz, dx, courant=0.99, cpml=None, stream=None):
        self._lib = _lib.load()
        self._h = None
        self.shape = (nz, ny, nx)
        self.nx, self.ny, self.nz, self.dx = nx, ny, nz, dx
        self._arena = None
        self.stream = stream
        cp = None
        if cpml:
            p = dict(cells=cpml) if isinstance(cpml, int) else dict(cpml)
            cp = CpmlParams(int(p["cells"]), float(p.get("order", 3.0)), float(p.get("kappa_max", 1.0)),
                            float(p.get("alpha_max", 0.0)), float(p.get("alpha_order", 1.0)),
                            float(p.get("sigma_max", 0.0)))
        h = ctypes.c_void_p()
        rc = self._lib.fdtd_create_grid(int(nx), int(ny), int(nz), float(dx), float(courant),
                                        ctypes.byref(cp) if cp else None, _stream_ptr(stream),
                                        ctypes.byref(h))
        check(self._lib, None, rc, "fdtd_create_grid")
        self._h = h
        self.probe_capacity = 0

    # -- lifetime --------------------------------------------------------
    def close(self):
        if self._h:
            self._lib.fdtd_destroy(self._h)
            self._h = None
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- description -----------------------------------------------------
    def set_materials(self, cell_material, table):
        cm = np.ascontiguousarray(cell_material, dtype=np.uint8)
        if cm.shape != self.shape:
            raise ValueError(f"material map shape {cm.shape} != {self.shape}")
        mats = (Material * len(table))(*[Material(float(e), float(s), float(m)) for e, s, m in table])
        check(self._lib, self._h, self._lib.fdtd_set_materials(
            self._h, cm.ctypes.data_as(ctypes.c_void_p), mats, len(table)), "set_materials")

    def set_debye(self, material, delta_eps, tau):
        """Debye poles (relative delta eps, tau in s; at most 4) of one
        material; its eps_r and sigma are eps_inf and the static sigma"""
        d = np.ascontiguousarray(delta_eps, dtype=np.float64)
        t = np.ascontiguousarray(tau, dtype=np.float64)
        if d.shape != t.shape:
            raise ValueError("delta_eps and tau differ in length")
        check(self._lib, self._h, self._lib.fdtd_set_debye(self._h, int(material), len(d),
                                                           d.ctypes.data_as(ctypes.c_void_p),
                                                           t.ctypes.data_as(ctypes.c_void_p)), "set_debye")

    def add_wire(self, p0, p1, radius):
        wid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_wire(self._h, *map(int, p0), *map(int, p1),
                                                          float(radius), ctypes.byref(wid)), "add_wire")
        return wid.value

    def add_wire_path(self, p0, p1, radius):
        """thin wire between two arbitrary nodes as a staircase of
        grid-aligned wires; returns the number of wires added"""
        n = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_wire_path(self._h, *map(int, p0), *map(int, p1),
                                                               float(radius), ctypes.byref(n)), "add_wire_path")
        return n.value

    def add_oblique_wire(self, p0, p1, radius):
        """oblique thin wire between two points in node units (any real
        coordinates); returns its id"""
        wid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_oblique_wire(self._h, *map(float, p0), *map(float, p1),
                                                                 float(radius), ctypes.byref(wid)),
              "add_oblique_wire")
        return wid.value

    def add_wire_voltage_source(self, wire, segment, voltage, r_internal=0.0):
        """delta-gap EMF (V at t_n) in one segment of an oblique wire, in
        series with r_internal ohm"""
        v = np.ascontiguousarray(voltage, dtype=np.float64)
        sid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_wire_voltage_source(
            self._h, int(wire), int(segment), float(r_internal), v.ctypes.data_as(ctypes.c_void_p), len(v),
            ctypes.byref(sid)), "add_wire_voltage_source")
        return sid.value

    def add_wire_probe(self, wire, segment):
        """current of one oblique-wire segment at t_{n+1/2}; returns the probe id"""
        pid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_wire_probe(self._h, int(wire), int(segment),
                                                               ctypes.byref(pid)), "add_wire_probe")
        return pid.value

    def add_wire_node_probe(self, point):
        """in-cell potential of the oblique-wire node at point (t_{n+1}); returns the probe id"""
        pid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_wire_node_probe(self._h, *map(float, point),
                                                                    ctypes.byref(pid)), "add_wire_node_probe")
        return pid.value

    def wire_counts(self):
        ns, nn = ctypes.c_int(), ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_wire_counts(self._h, ctypes.byref(ns), ctypes.byref(nn)),
              "wire_counts")
        return ns.value, nn.value

    def wire_courant_limit(self):
        """largest Courant number the oblique wires added so far allow"""
        c = ctypes.c_double()
        check(self._lib, self._h, self._lib.fdtd_wire_courant_limit(self._h, ctypes.byref(c)),
              "wire_courant_limit")
        return c.value

    def get_wire_state(self):
        """(segment currents of the last half step, node charges)"""
        ns, nn = self.wire_counts()
        I, Q = np.zeros(max(ns, 1), np.float32), np.zeros(max(nn, 1), np.float32)
        check(self._lib, self._h, self._lib.fdtd_get_wire_state(self._h, I.ctypes.data_as(ctypes.c_void_p),
                                                               Q.ctypes.data_as(ctypes.c_void_p)), "get_wire_state")
        return I[:ns], Q[:nn]

    def set_wire_state(self, I, Q):
        ns, nn = self.wire_counts()
        I = np.ascontiguousarray(I, dtype=np.float32)
        Q = np.ascontiguousarray(Q, dtype=np.float32)
        if I.shape != (ns,) or Q.shape != (nn,):
            raise ValueError("wire state shapes do not match the wire counts")
        check(self._lib, self._h, self._lib.fdtd_set_wire_state(self._h, I.ctypes.data_as(ctypes.c_void_p),
                                                               Q.ctypes.data_as(ctypes.c_void_p)), "set_wire_state")

    def add_source(self, node, axis, current, r_internal=0.0):
        cur = np.ascontiguousarray(current, dtype=np.float64)
        sid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_source(
            self._h, *map(int, node), int(axis), float(r_internal), cur.ctypes.data_as(ctypes.c_void_p),
            len(cur), ctypes.byref(sid)), "add_source")
        return sid.value

    def add_voltage_source(self, node, axis, voltage, r_internal=0.0):
        """voltage source V = -E dx across the edge: ideal (r_internal = 0,
        voltage[n] at t_{n+1}) or in series with r_internal (at t_{n+1/2})"""
        v = np.ascontiguousarray(voltage, dtype=np.float64)
        sid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_voltage_source(
            self._h, *map(int, node), int(axis), float(r_internal), v.ctypes.data_as(ctypes.c_void_p), len(v),
            ctypes.byref(sid)), "add_voltage_source")
        return sid.value

    def add_lumped(self, node, axis, resistance=0.0, capacitance=0.0):
        lid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_lumped(self._h, *map(int, node), int(axis), float(resistance),
                                                            float(capacitance), ctypes.byref(lid)), "add_lumped")
        return lid.value

    def add_probe(self, kind, node, axis, n_edges=1):
        pid = ctypes.c_int()
        check(self._lib, self._h, self._lib.fdtd_add_probe(self._h, int(kind), *map(int, node), int(axis),
                                                           int(n_edges), ctypes.byref(pid)), "add_probe")
        return pid.value

    def set_block(self, planes):
        """planes per work item of the step kernel (tuning; 0 = default)"""
        check(self._lib, self._h, self._lib.fdtd_set_block(self._h, int(planes)), "set_block")

    def set_watchdog(self, every):
        """divergence watchdog period in steps (0 = off): synchronising
        calls raise FdtdError(FDTD_EDIVERGED) after a check that found a NaN
        or an infinity"""
        check(self._lib, self._h, self._lib.fdtd_set_watchdog(self._h, int(every)), "set_watchdog")

    def arena_bytes(self, probe_capacity):
        b = ctypes.c_size_t()
        check(self._lib, self._h, self._lib.fdtd_arena_bytes(self._h, int(probe_capacity), ctypes.byref(b)),
              "arena_bytes")
        return b.value

    def finalize(self, probe_capacity=0, torch_arena=True):
        """Build classes and upload.  With torch_arena the device memory is
        one torch uint8 tensor owned by this object."""
        ptr, nbytes = None, 0
        if torch_arena:
            import torch
            nbytes = self.arena_bytes(probe_capacity)
            self._arena = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._arena.data_ptr()
            ptr = ctypes.c_void_p((base + 255) // 256 * 256)
        check(self._lib, self._h, self._lib.fdtd_finalize(self._h, int(probe_capacity), ptr, nbytes),
              "finalize")
        self.probe_capacity = int(probe_capacity)

    # -- running ---------------------------------------------------------
    def step(self, n=1):
        check(self._lib, self._h, self._lib.fdtd_step(self._h, int(n)), "step")

    def step_noalloc(self, n=1):
        """n steps through fdtd_step_noalloc (no device allocation; the step
        kernel's scratch is a static device array shared by all such calls)."""
        check(self._lib, self._h, self._lib.fdtd_step_noalloc(self._h, int(n)), "step_noalloc")

    def synchronize(self):
        check(self._lib, self._h, self._lib.fdtd_synchronize(self._h), "synchronize")

    def read_probe(self, probe_id, first=0, count=None):
        if count is None:
            count = self.probe_capacity - first
        out = np.empty(max(count, 0), dtype=np.float32)
        check(self._lib, self._h, self._lib.fdtd_read_probes(
            self._h, int(probe_id), int(first), int(count), out.ctypes.data_as(ctypes.c_void_p)), "read_probes")
        return out

    def get_field(self, comp):
        out = np.empty(self.shape, dtype=np.float32)
        check(self._lib, self._h, self._lib.fdtd_get_field(self._h, int(comp),
                                                           out.ctypes.data_as(ctypes.c_void_p)), "get_field")
        return out

    def set_field(self, comp, values):
        v = np.ascontiguousarray(values, dtype=np.float32)
        if v.shape != self.shape:
            raise ValueError(f"field shape {v.shape} != {self.shape}")
        check(self._lib, self._h, self._lib.fdtd_set_field(self._h, int(comp), v.ctypes.data_as(ctypes.c_void_p)),
              "set_field")

    def save_state(self):
        """the grid's checkpoint (fields, CPML auxiliaries, probe record,
        step count) as bytes"""
        n = ctypes.c_size_t()
        check(self._lib, self._h, self._lib.fdtd_save_state(self._h, None, ctypes.byref(n)), "save_state")
        buf = ctypes.create_string_buffer(n.value)
        check(self._lib, self._h, self._lib.fdtd_save_state(self._h, buf, ctypes.byref(n)), "save_state")
        return buf.raw[:n.value]

    def load_state(self, state):
        check(self._lib, self._h, self._lib.fdtd_load_state(self._h, state, len(state)), "load_state")

    def field_device(self, comp):
        p = ctypes.c_void_p()
        rp = ctypes.c_int()
        pp = ctypes.c_size_t()
        check(self._lib, self._h, self._lib.fdtd_field_device(self._h, int(comp), ctypes.byref(p),
                                                              ctypes.byref(rp), ctypes.byref(pp)), "field_device")
        return p.value, rp.value, pp.value

    @property
    def dt(self):
        return self._lib.fdtd_get_dt(self._h)

    @property
    def step_count(self):
        return self._lib.fdtd_get_step(self._h)

    @property
    def num_classes(self):
        return self._lib.fdtd_num_classes(self._h)


class Batch:
    """Advance many finalized grids together (the batched engine of the C
    ABI): one persistent launch per step over all domains, graph-replayed."""

    def __init__(self, grids, stream=None):
        self._lib = _lib.load()
        self.grids = list(grids)
        arr = (ctypes.c_void_p * len(self.grids))(*[g._h for g in self.grids])
        h = ctypes.c_void_p()
        rc = self._lib.fdtd_batch_create(len(self.grids), arr, _stream_ptr(stream), ctypes.byref(h))
        if rc != 0:
            raise FdtdError(rc, "fdtd_batch_create")
        self._h = h

    def _check(self, rc, what):
        if rc != 0:
            raise FdtdError(rc, f"{what}: {self._lib.fdtd_batch_last_error(self._h).decode()}")

    def step(self, n=1):
        self._check(self._lib.fdtd_batch_step(self._h, int(n)), "batch_step")

    def synchronize(self):
        self._check(self._lib.fdtd_batch_synchronize(self._h), "batch_synchronize")

    def launch_info(self, launch):
        c, i = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.fdtd_batch_launch_info(self._h, int(launch), ctypes.byref(c), ctypes.byref(i)),
                    "batch_launch_info")
        return c.value, i.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fdtd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_scenario(sc, stream=None, probe_capacity=None, torch_arena=True, block=0):
    """Build and finalize a Grid from a workloads.Scenario."""
    g = Grid(*sc.n, sc.dx, courant=sc.courant, cpml=sc.cpml or None, stream=stream)
    if block:
        g.set_block(block)
    g.set_materials(sc.cell_material, sc.materials)
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
    g.finalize(sc.n_steps if probe_capacity is None else probe_capacity, torch_arena=torch_arena)
    return g


__all__ = ["Grid", "Batch", "FdtdError", "from_scenario", "EX", "EY", "EZ", "HX", "HY", "HZ",
           "PROBE_V", "PROBE_I", "PROBE_E", "PROBE_H", "PROBE_WIRE", "PROBE_WIRE_V"]
