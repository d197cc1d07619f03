"""Test helpers: run a workloads.Scenario on the oracle and compare results."""
import numpy as np

from oracle.oracle import OracleGrid


def oracle_from_scenario(sc, parity=True):
    return OracleGrid.from_scenario(sc, parity=parity)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ---- record of achieved parity errors ---------------------------------------
# When FDTD_PARITY_RECORD names a file, every comparison that goes through
# record() appends one JSON line to it: the case, the quantity compared, the
# relative L2 error achieved, the bar it was held to and, for runs from rest,
# the error of the same algorithm with FP32 storage (the yardstick of the
# from-rest bar).  tests/parity_summary.py turns the file into a table.
def record(case, quantity, err, bar, fp32_yardstick=None, steps=None, norm=None):
    import json
    import os
    path = os.environ.get("FDTD_PARITY_RECORD")
    if not path:
        return
    if case is None:
        case = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0].split("::")[-1]
    line = {"case": case, "quantity": quantity, "rel_l2": float(err), "bar": float(bar),
            "stated_bar": 1e-5 if quantity.startswith("field") else 1e-4}
    if fp32_yardstick is not None:
        line["fp32_yardstick"] = float(fp32_yardstick)
    if steps is not None:
        line["steps"] = int(steps)
    if norm is not None:
        line["relative_to"] = norm
    with open(path, "a") as f:
        f.write(json.dumps(line) + "\n")


COMPONENTS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")


def field_errors(got, ref, vanish=1e-6):
    """Relative L2 error of each of the six components (Ex Ey Ez Hx Hy Hz)
    of got against ref.  A component whose reference is below `vanish` times
    the norm of its vector field (E or H) is zero in exact arithmetic (e.g.
    Hz of a vertical source on a vertical wire in horizontally layered
    media, a TM field): its reference is FP64 roundoff, so its error is
    taken relative to the norm of the whole vector field instead.
    Returns [(error, 'component' | 'vector field')] * 6."""
    out = []
    for v in (0, 3):
        vec = np.sqrt(sum(np.linalg.norm(np.asarray(ref[c], np.float64)) ** 2 for c in range(v, v + 3)))
        for c in range(v, v + 3):
            r = np.asarray(ref[c], np.float64)
            nr = np.linalg.norm(r)
            d = np.linalg.norm(np.asarray(got[c], np.float64) - r)
            if vec > 0 and nr < vanish * vec:
                out.append((d / vec, "vector field"))
            else:
                out.append((d / (nr if nr > 0 else 1.0), "component"))
    return out
