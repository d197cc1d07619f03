"""Build the CUDA library in-tree with nvcc for sm_103a.

The translation units under csrc/ compile in parallel to objects, then link
into ``_build/libfdtd_gb300.so`` next to this file.  No CPU fallback is
built: the library is the only implementation of the path.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libfdtd_gb300.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-fast-math",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


BOUNDS_LIB = os.path.join(BUILD, "bounds", "libfdtd_gb300.so")


def build_bounds(force: bool = False) -> str:
    """The bounds-checked build (a debugging aid, not the product path):
    the same sources compiled with -DFDTD_BOUNDS into _build/bounds/, where
    every global access of the step and source/probe kernels tests its index
    (fdtd_bounds_report reads the record).  Load it by setting FDTD_LIBRARY
    to the returned path before the binding loads the library."""
    return build(force=force, extra=["-DFDTD_BOUNDS"], lib=BOUNDS_LIB)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, lib: str = LIB) -> str:
    if not force and up_to_date(lib):
        return lib
    bdir = os.path.dirname(lib)
    os.makedirs(bdir, exist_ok=True)
    extra = list(extra or [])
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(cmd[-3])
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(failed))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
