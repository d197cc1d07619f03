"""The boundary from plain C: include/fdtd.h and include/fdtd_mlp.h compile
as C99 with warnings as errors, a C program links the library and its
host-side calls behave as documented (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_2207_06908_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_c_program_uses_the_abi(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    lib = _build.build()
    exe = tmp_path / "c_abi_host"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", _build.INCLUDE,
           os.path.join(HERE, "c_abi_host.c"), "-L", os.path.dirname(lib), "-lfdtd_gb300",
           "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok "), r.stdout + r.stderr
