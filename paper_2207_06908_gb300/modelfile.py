"""Plain-text model files: the command language of the paper's command-line
program (Kuklin, arXiv 2207.06908, Sec. 3 "Interface", and the model files
of Sec. 4), read into a workloads.Scenario that runs on the GB300 library
(fdtd.from_scenario).

One command per line, ``name (arg, arg, ...)``; lengths in metres, times in
seconds; text after ``#`` or ``%`` is a comment.  The paper names the
commands and shows them in use but defines few of their arguments; where it
is silent this reader takes the reading stated beside the command:

  volume (X, Y, Z, dx)
      round(X/dx) x round(Y/dx) x round(Z/dx) cells of size dx.
  calctime (T)
      ceil(T/dt) steps, dt = S dx / (c0 sqrt 3) at the Courant number S
      given to parse() (0.99 by default).
  output (dt_out)
      the probes' output interval, kept in Model.output_dt (see
      Model.resample); the library records every step.
  abc (cpml, thickness, ...)
      a CPML of round(thickness/dx) cells with the library's profile (cubic
      grading, kappa_max 1, alpha 0); the further arguments are not read.
  block (x0, y0, z0, x1, y1, z1, eps_r, sigma [, debye])
      the cells whose centres lie in the box take the medium (relative
      permittivity, conductivity in S/m, mu_r 1, the named Debye poles);
      later blocks override earlier ones; the rest is air.
  debye (name, deps1, tau1 [, deps2, tau2, ...])
      up to four poles (relative deps, tau in s) for blocks naming it.
  wire (thin, x0, y0, z0, x1, y1, z1, radius [, t])
      a thin wire between two points: along a node line, the modified-
      coefficient wire (Sec. 2.3); otherwise an oblique wire; a trailing
      flag is ignored.  ``wire (oblique, ...)`` and ``wire (staircase, ...)``
      choose a model explicitly.
  source (current, x0, y0, z0, x1, y1, z1, r, fn)
      a current source on the one-cell edge between the two nodes, current
      positive from the first point to the second, internal resistance r
      (0 = ideal), waveform the function fn.
  calculate (current | voltage, x0, y0, z0, x1, y1, z1)
      a probe: the loop current around the one-cell edge between the nodes
      (positive from the first to the second), or the voltage -sum E dl
      along the straight node path from the first point to the second.
  function (fn, custom, dt, v0, v1, ...)
      samples v_q at t = q dt, linear in between, 0 after the last.
  function (fn, heidler, mode, tau1, tau2, i0, n [, eta, t0])
      i0 / eta (s^n / (1 + s^n)) exp(-(t - t0) / tau2), s = (t - t0) / tau1,
      for t > t0; eta <= 0 or absent: the peak correction that makes the
      peak i0; the mode word is not read.
  function (fn, ramp, i0, t_rise) / function (fn, dexp, i0, alpha, beta)
      a linear rise to i0, held; i0 (exp(-alpha t) - exp(-beta t)).

Sources are sampled at t_{n+1/2}.  Errors raise ValueError naming the line.
"""
from __future__ import annotations

import dataclasses
import math
import re
import sys

import numpy as np

from . import workloads as W

_CMD = re.compile(r"^\s*([A-Za-z_]\w*)\s*\((.*)\)\s*$")


@dataclasses.dataclass
class Model:
    scenario: W.Scenario
    output_dt: float | None          # probe output interval (output command), None: every step
    probe_names: list                # ("current" | "voltage", line, sign) per probe, in probe order;
                                     # sign -1: the file's orientation is against +axis

    def resample(self, samples: np.ndarray, kind: str = "current") -> tuple:
        """probe samples of every step -> (times, values) at the output
        interval, linear in between; currents are recorded at t_{n+1/2},
        voltages at t_{n+1}"""
        dt = W.time_step(self.scenario.dx, self.scenario.courant)
        t = (np.arange(len(samples)) + (0.5 if kind == "current" else 1.0)) * dt
        if not self.output_dt:
            return t, np.asarray(samples)
        to = np.arange(0.0, t[-1] + 1e-30, self.output_dt)
        return to, np.interp(to, t, samples, left=0.0)


def _split(args: str) -> list:
    return [a.strip() for a in args.split(",") if a.strip() != ""]


def _num(tok: str, line: int) -> float:
    try:
        return float(tok)
    except ValueError:
        raise ValueError(f"line {line}: '{tok}' is not a number") from None


def _waveform(spec: list, t: np.ndarray, line: int) -> np.ndarray:
    kind = spec[0].lower()
    v = spec[1:]
    if kind == "custom":
        if len(v) < 2:
            raise ValueError(f"line {line}: custom function needs an interval and samples")
        dt = _num(v[0], line)
        s = np.array([_num(x, line) for x in v[1:]])
        ts = np.arange(len(s)) * dt
        return np.interp(t, ts, s, left=s[0], right=0.0)
    if kind == "heidler":
        nums = [_num(x, line) for x in v[1:]]          # v[0]: the mode word
        if not 4 <= len(nums) <= 6:
            raise ValueError(f"line {line}: heidler takes tau1, tau2, i0, n [, eta, t0]")
        tau1, tau2, i0, n = nums[:4]
        eta = nums[4] if len(nums) > 4 else 0.0
        t0 = nums[5] if len(nums) > 5 else 0.0
        if eta <= 0.0:
            eta = math.exp(-(tau1 / tau2) * (n * tau2 / tau1) ** (1.0 / n))
        s = np.where(t > t0, (t - t0) / tau1, 0.0) ** n
        return np.where(t > t0, i0 / eta * s / (1.0 + s) * np.exp(-np.maximum(t - t0, 0.0) / tau2), 0.0)
    if kind == "ramp":
        if len(v) != 2:
            raise ValueError(f"line {line}: ramp takes i0, t_rise")
        i0, tr = (_num(x, line) for x in v)
        return W.ramp(t, i0, tr)
    if kind == "dexp":
        if len(v) != 3:
            raise ValueError(f"line {line}: dexp takes i0, alpha, beta")
        i0, a, b = (_num(x, line) for x in v)
        return i0 * (np.exp(-a * t) - np.exp(-b * t))
    raise ValueError(f"line {line}: unknown function type '{spec[0]}'")


def _node(p, dx, line, what):
    q = [c / dx for c in p]
    r = [round(c) for c in q]
    if any(abs(a - b) > 1e-6 for a, b in zip(q, r)):
        raise ValueError(f"line {line}: {what} point {tuple(p)} is not on a grid node")
    return r


def _edge(p0, p1, dx, line, what):
    """node, axis and sign (+1 from p0 to p1 along +axis) of a straight node path"""
    a, b = _node(p0, dx, line, what), _node(p1, dx, line, what)
    d = [y - x for x, y in zip(a, b)]
    axes = [u for u in range(3) if d[u] != 0]
    if len(axes) != 1:
        raise ValueError(f"line {line}: {what} must run along one axis between two different nodes")
    u = axes[0]
    lo = list(a) if d[u] > 0 else list(b)
    return tuple(lo), u, abs(d[u]), (1 if d[u] > 0 else -1)


def parse(text: str, courant: float = 0.99, name: str = "model") -> Model:
    """Read a model file into a Model (scenario, output interval, probes)."""
    cmds = []
    for ln, raw in enumerate(text.splitlines(), 1):
        s = re.split(r"[#%]", raw, maxsplit=1)[0].strip()
        if not s:
            continue
        m = _CMD.match(s)
        if not m:
            raise ValueError(f"line {ln}: expected 'command (arguments)'")
        cmds.append((ln, m.group(1).lower(), _split(m.group(2))))
    vol = [c for c in cmds if c[1] == "volume"]
    if len(vol) != 1:
        raise ValueError("a model file needs exactly one volume command")
    ln, _, a = vol[0]
    if len(a) != 4:
        raise ValueError(f"line {ln}: volume takes X, Y, Z, dx")
    X, Y, Z, dx = (_num(x, ln) for x in a)
    if not dx > 0:
        raise ValueError(f"line {ln}: the cell size must be positive")
    n = tuple(int(round(v / dx)) for v in (X, Y, Z))
    if min(n) < 2:
        raise ValueError(f"line {ln}: the volume must span at least two cells per axis")
    dt = W.time_step(dx, courant)
    n_steps, output_dt, cpml = 0, None, 0
    debye, funcs = {}, {}
    for ln, c, a in cmds:
        if c == "debye":
            if len(a) < 3 or len(a) % 2 == 0 or len(a) > 9:
                raise ValueError(f"line {ln}: debye takes a name and one to four (deps, tau) pairs")
            v = [_num(x, ln) for x in a[1:]]
            debye[a[0]] = (v[0::2], v[1::2])
        elif c == "function":
            if len(a) < 3:
                raise ValueError(f"line {ln}: function takes a name, a type and parameters")
            funcs[a[0]] = (a[1:], ln)
        elif c == "calctime":
            n_steps = int(math.ceil(_num(a[0], ln) / dt - 1e-9))
        elif c == "output":
            output_dt = _num(a[0], ln)
        elif c == "abc":
            if not a or a[0].lower() != "cpml" or len(a) < 2:
                raise ValueError(f"line {ln}: only abc (cpml, thickness, ...) is supported")
            cpml = int(round(_num(a[1], ln) / dx))
    if n_steps <= 0:
        raise ValueError("a model file needs a positive calctime")
    t_src = W.sample_times(n_steps, dx, courant)

    cm = np.zeros((n[2], n[1], n[0]), np.uint8)
    materials = [(1.0, 0.0, 1.0)]
    mat_debye = {}
    keys = {(1.0, 0.0, None): 0}
    wires, owires, paths, sources, probes, names = [], [], [], [], [], []
    for ln, c, a in cmds:
        if c == "block":
            if len(a) not in (8, 9):
                raise ValueError(f"line {ln}: block takes x0, y0, z0, x1, y1, z1, eps_r, sigma [, debye]")
            v = [_num(x, ln) for x in a[:8]]
            deb = a[8] if len(a) == 9 else None
            if deb is not None and deb not in debye:
                raise ValueError(f"line {ln}: no debye command named '{deb}'")
            key = (v[6], v[7], deb)
            if key not in keys:
                if len(materials) == 256:
                    raise ValueError(f"line {ln}: more than 256 media")
                keys[key] = len(materials)
                materials.append((v[6], v[7], 1.0))
                if deb is not None:
                    mat_debye[keys[key]] = debye[deb]
            lo = [max(0, math.ceil(v[u] / dx - 0.5)) for u in range(3)]
            hi = [min(n[u], math.floor(v[3 + u] / dx - 0.5) + 1) for u in range(3)]
            if all(h > l for l, h in zip(lo, hi)):
                cm[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = keys[key]
        elif c == "wire":
            if len(a) not in (8, 9):
                raise ValueError(f"line {ln}: wire takes a model, two points, a radius [, flag]")
            model = a[0].lower()
            v = [_num(x, ln) for x in a[1:8]]
            p0, p1, r = v[0:3], v[3:6], v[6]
            # node units, snapped to 1e-9 cell: decimal metres give the intended points
            q0, q1 = [round(x / dx, 9) for x in p0], [round(x / dx, 9) for x in p1]
            on_grid = all(abs(x - round(x)) < 1e-6 for x in q0 + q1)
            aligned = sum(abs(x - y) > 1e-9 for x, y in zip(q0, q1)) == 1
            if model == "thin" and on_grid and aligned:
                node, u, length, _ = _edge(p0, p1, dx, ln, "wire")
                end = list(node)
                end[u] += length
                wires.append((tuple(node), tuple(end), r))
            elif model in ("thin", "oblique"):
                owires.append((tuple(q0), tuple(q1), r))
            elif model == "staircase":
                paths.append((tuple(_node(p0, dx, ln, "wire")), tuple(_node(p1, dx, ln, "wire")), r))
            else:
                raise ValueError(f"line {ln}: unknown wire model '{a[0]}'")
        elif c == "source":
            if len(a) != 9 or a[0].lower() != "current":
                raise ValueError(f"line {ln}: source takes current, two points, r, function")
            v = [_num(x, ln) for x in a[1:8]]
            node, u, length, sign = _edge(v[0:3], v[3:6], dx, ln, "source")
            if length != 1:
                raise ValueError(f"line {ln}: a source spans one cell")
            if a[8] not in funcs:
                raise ValueError(f"line {ln}: no function named '{a[8]}'")
            spec, fl = funcs[a[8]]
            cur = sign * _waveform(spec, t_src, fl)
            sources.append((node, u, cur, v[6]) if v[6] > 0 else (node, u, cur))
        elif c == "calculate":
            if len(a) != 7 or a[0].lower() not in ("current", "voltage"):
                raise ValueError(f"line {ln}: calculate takes current or voltage and two points")
            v = [_num(x, ln) for x in a[1:7]]
            node, u, length, sign = _edge(v[0:3], v[3:6], dx, ln, "probe")
            if a[0].lower() == "current":
                if length != 1:
                    raise ValueError(f"line {ln}: a current probe spans one cell")
                probes.append((W.PROBE_I, node, u, 1))
            else:
                probes.append((W.PROBE_V, node, u, length))
            names.append((a[0].lower(), ln, sign))
        elif c not in ("volume", "calctime", "output", "abc", "debye", "function"):
            raise ValueError(f"line {ln}: unknown command '{c}'")
    sc = W.Scenario(name, n, dx, courant, cpml, cm, materials, wires=wires, sources=sources, probes=probes,
                    n_steps=n_steps)
    sc.debye = mat_debye
    sc.owires = owires
    sc.wire_paths = paths
    return Model(sc, output_dt, names)


def load(path: str, courant: float = 0.99) -> Model:
    with open(path) as f:
        return parse(f.read(), courant=courant, name=path)


def run(model: Model):
    """Run a model on the GPU; returns [(kind, times, values)] per probe, at
    the output interval, each probe read with its stated orientation."""
    from . import fdtd
    sc = model.scenario
    g = fdtd.from_scenario(sc, probe_capacity=sc.n_steps)
    g.step(sc.n_steps)
    out = []
    for p, (kind, _, sign) in enumerate(model.probe_names):
        t, v = model.resample(sign * g.read_probe(p), kind)
        out.append((kind, t, v))
    g.close()
    return out


def main(argv=None) -> int:
    import argparse
    ap = argparse.ArgumentParser(description="run a model file on the GPU and print the probes as CSV")
    ap.add_argument("model")
    ap.add_argument("--courant", type=float, default=0.99)
    ap.add_argument("--parse-only", action="store_true", help="check the file and print its size")
    a = ap.parse_args(argv)
    m = load(a.model, a.courant)
    sc = m.scenario
    if a.parse_only:
        print(f"{sc.n[0]}x{sc.n[1]}x{sc.n[2]} cells, dx {sc.dx} m, {sc.n_steps} steps, CPML {sc.cpml}, "
              f"{len(sc.materials)} media, {len(sc.wires)} thin + {len(sc.owires)} oblique + "
              f"{len(sc.wire_paths)} staircase wires, {len(sc.sources)} sources, {len(sc.probes)} probes")
        return 0
    res = run(m)
    if not res:
        return 0
    print("t," + ",".join(f"{k}{i}" for i, (k, _, _) in enumerate(res)))
    n = min(len(t) for _, t, _ in res)
    for q in range(n):
        print(f"{res[0][1][q]:.6e}," + ",".join(f"{v[q]:.6e}" for _, _, v in res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
