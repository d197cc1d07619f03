"""Batched grounding runs: build many grounding-electrode domains, advance
them together with the batched engine of the C ABI, and return each
domain's transient impedance waveform (gap voltage over peak current at 512
uniform instants).  Marshalling and host-side bookkeeping only; every step
runs in the CUDA library.

The tile depth (planes per work item) of each domain comes from a small
autotuner: for each 16-cell size class it times the candidates on a batch of
copies of a representative domain (the regime the depth serves) once and
keeps the winners in a JSON cache in the build folder.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import fdtd, workloads as W

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")
CANDIDATES = (8, 12, 16, 24, 32, 48)


def size_class(n: int) -> int:
    """domains are tuned per 16-cell size class"""
    return (n + 15) // 16 * 16


def _load_cache():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(c):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def tune_block(n: int, steps: int = 32, force: bool = False) -> int:
    """Planes per work item for n^3 grounding domains advanced in a batch:
    the candidate with the shortest measured step of a batch of copies of a
    representative domain (enough copies that the batch, not one domain,
    fills the GPU, as in the batches this serves; cached)."""
    import torch
    key = f"ground_batch_n{size_class(n)}"
    cache = _load_cache()
    if key in cache and not force:
        return int(cache[key])
    m = size_class(n)
    copies = int(max(8, min(64, 4.0e7 // m ** 3)))
    sc = W.grounding_domain(m, 15.0, 1e-3, 1.0, 0.008, 0.0, 0.25e-6, n_steps=steps + 8)
    best, best_t = 8, float("inf")
    for kz in CANDIDATES:
        if kz > m:
            continue
        grids = [fdtd.from_scenario(sc, probe_capacity=steps + 8, block=kz) for _ in range(copies)]
        b = fdtd.Batch(grids)
        b.step(8)
        b.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        b.step(steps)
        e1.record(s)
        b.synchronize()
        t = e0.elapsed_time(e1)
        b.close()
        for g in grids:
            g.close()
        if t < best_t:
            best, best_t = kz, t
    cache[key] = best
    _store_cache(cache)
    return best


def run_batch(scenarios, tuned: bool = True, timings: dict | None = None):
    """Advance every scenario for its n_steps (all equal) as one batch;
    returns (waveforms [n, 512], probe traces list).  timings, if given,
    receives setup / step / readback seconds and the device step time."""
    import torch
    steps = scenarios[0].n_steps
    assert all(sc.n_steps == steps for sc in scenarios)
    t0 = time.perf_counter()
    blocks = {}
    if tuned:
        for sc in scenarios:
            c = size_class(sc.n[0])
            if c not in blocks:
                blocks[c] = tune_block(sc.n[0])
    grids = [fdtd.from_scenario(sc, probe_capacity=steps, block=blocks.get(size_class(sc.n[0]), 0))
             for sc in scenarios]
    b = fdtd.Batch(grids)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    b.step(steps)
    e1.record(s)
    b.synchronize()
    t2 = time.perf_counter()
    traces = [[g.read_probe(p, 0, steps) for p in range(len(sc.probes))] for g, sc in zip(grids, scenarios)]
    dt = grids[0].dt
    waves = np.stack([W.impedance_waveform(tr[0], dt) for tr in traces])
    t3 = time.perf_counter()
    if timings is not None:
        timings.update(setup_s=t1 - t0, step_s=t2 - t1, readback_s=t3 - t2, device_ms=e0.elapsed_time(e1),
                       ctas=[b.launch_info(0), b.launch_info(1)])
    b.close()
    for g in grids:
        g.close()
    return waves, traces
