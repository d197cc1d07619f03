"""ctypes binding of the C ABI in include/fdtd.h (argument marshalling only).

Every step of the path runs in the CUDA library; there is no CPU fallback.
Loading fails with an exception when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

_lock = threading.Lock()
_lib = None

FDTD_OK = 0
ERRORS = {
    -1: "FDTD_EINVAL", -2: "FDTD_ECOURANT", -3: "FDTD_ENOMEM", -4: "FDTD_ECUDA",
    -5: "FDTD_ECLASSES", -6: "FDTD_ETIMEOUT", -7: "FDTD_EDIVERGED", -8: "FDTD_ESTATE",
}


class FdtdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class CpmlParams(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int), ("order", ctypes.c_double), ("kappa_max", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("alpha_order", ctypes.c_double),
                ("sigma_max", ctypes.c_double)]


class Material(ctypes.Structure):
    _fields_ = [("eps_r", ctypes.c_double), ("sigma", ctypes.c_double), ("mu_r", ctypes.c_double)]


def lib_path() -> str:
    """the release library, or the build FDTD_LIBRARY names (the
    bounds-checked build of _build.build_bounds)"""
    return os.environ.get("FDTD_LIBRARY") or _build.LIB


def load():
    """Load libfdtd_gb300.so (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build() or python -m paper_2207_06908_gb300._build)")
        lib = ctypes.CDLL(path)
        P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        ip = ctypes.POINTER(ctypes.c_int)
        sig = {
            "fdtd_create_grid": (I, [I, I, I, D, D, ctypes.POINTER(CpmlParams), P, ctypes.POINTER(P)]),
            "fdtd_set_materials": (I, [P, P, ctypes.POINTER(Material), I]),
            "fdtd_add_wire": (I, [P, I, I, I, I, I, I, D, ip]),
            "fdtd_add_source": (I, [P, I, I, I, I, D, P, I, ip]),
            "fdtd_add_probe": (I, [P, I, I, I, I, I, I, ip]),
            "fdtd_set_block": (I, [P, I]),
            "fdtd_set_watchdog": (I, [P, I]),
            "fdtd_bounds_report": (I, [P, ip, ip]),
            "fdtd_arena_bytes": (I, [P, I, ctypes.POINTER(S)]),
            "fdtd_finalize": (I, [P, I, P, S]),
            "fdtd_step": (I, [P, I]),
            "fdtd_step_noalloc": (I, [P, I]),
            "fdtd_synchronize": (I, [P]),
            "fdtd_read_probes": (I, [P, I, I, I, P]),
            "fdtd_get_field": (I, [P, I, P]),
            "fdtd_set_field": (I, [P, I, P]),
            "fdtd_field_device": (I, [P, I, ctypes.POINTER(P), ip, ctypes.POINTER(S)]),
            "fdtd_get_dt": (D, [P]),
            "fdtd_get_step": (ctypes.c_long, [P]),
            "fdtd_num_classes": (I, [P]),
            "fdtd_last_error": (ctypes.c_char_p, [P]),
            "fdtd_destroy": (None, [P]),
            "fdtd_batch_create": (I, [I, P, P, ctypes.POINTER(P)]),
            "fdtd_batch_step": (I, [P, I]),
            "fdtd_batch_synchronize": (I, [P]),
            "fdtd_batch_launch_info": (I, [P, I, ip, ip]),
            "fdtd_batch_last_error": (ctypes.c_char_p, [P]),
            "fdtd_batch_destroy": (None, [P]),
            "fdtd_selftest_wait": (I, [ctypes.c_double, P]),
            "fdtd_set_debye": (I, [P, I, I, P, P]),
            "fdtd_add_voltage_source": (I, [P, I, I, I, I, ctypes.c_double, P, I, P]),
            "fdtd_add_lumped": (I, [P, I, I, I, I, ctypes.c_double, ctypes.c_double, P]),
            "fdtd_add_wire_path": (I, [P, I, I, I, I, I, I, ctypes.c_double, P]),
            "fdtd_add_oblique_wire": (I, [P, D, D, D, D, D, D, D, ip]),
            "fdtd_add_wire_voltage_source": (I, [P, I, I, D, P, I, ip]),
            "fdtd_add_wire_probe": (I, [P, I, I, ip]),
            "fdtd_add_wire_node_probe": (I, [P, D, D, D, ip]),
            "fdtd_wire_counts": (I, [P, ip, ip]),
            "fdtd_wire_courant_limit": (I, [P, ctypes.POINTER(D)]),
            "fdtd_get_wire_state": (I, [P, P, P]),
            "fdtd_set_wire_state": (I, [P, P, P]),
            "fdtd_save_state": (I, [P, P, ctypes.POINTER(ctypes.c_size_t)]),
            "fdtd_load_state": (I, [P, P, ctypes.c_size_t]),
            "fdtd_mlp_forward": (I, [P, I, I, I, P, P, I, I, P, P, P, P]),
            "fdtd_mlp_backward": (I, [P, I, P, P, I, I, I, I, P, P, P, P, P, P]),
            "fdtd_mlp_adam": (I, [P, P, P, P, P, I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_float, I, P]),
            "fdtd_mlp_mse": (I, [P, P, P, I, I, ctypes.c_float, P, P, P]),
            "fdtd_mlp_row_rel_err": (I, [P, P, I, I, P, P]),
            "fdtd_mlp_gather_rows": (I, [P, P, I, I, P, P]),
            "fdtd_mlp_scale_rows": (I, [P, P, I, I, P]),
            "fdtd_mlp_to_bf16": (I, [P, P, I, P]),
            "fdtd_mlp_check": (I, [P]),
            "fdtd_mlp_net_pack_bytes": (I, [ip, I, ctypes.POINTER(S)]),
            "fdtd_mlp_net_pack": (I, [ip, I, ctypes.POINTER(P), P, P]),
            "fdtd_mlp_net_forward": (I, [P, I, ip, I, ip, P, ctypes.POINTER(P), ctypes.c_float, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(lib, handle, rc: int, what: str):
    if rc != FDTD_OK:
        msg = lib.fdtd_last_error(handle).decode() if handle else what
        raise FdtdError(rc, f"{what}: {msg}")
