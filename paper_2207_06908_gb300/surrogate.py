"""Learned surrogate of the grounding-electrode runs: a multilayer perceptron
6 -> 256 -> 256 -> 256 -> 512 (GELU) mapping (eps_r, log10 sigma, rod length,
rod radius, burial depth, current rise time) to the 512-sample transient
impedance waveform that the batched FDTD engine produces for the same
parameters, plus a small error head that predicts the network's relative L2
error so that uncertain inputs fall back to FDTD.

The paper has no learned component; the surrogate is an addition built on the
paper's grounding-electrode model (its ground-potential-rise example: rod,
riser, current and voltage leads into the absorbing boundary).  Dataset
generation, training and inference all run in this library's CUDA kernels
(the FDTD engine of include/fdtd.h and the BF16 tensor-core layers of
include/fdtd_mlp.h); this module only marshals arrays and keeps host-side
bookkeeping.
"""
from __future__ import annotations

import time

import numpy as np

from . import fdtd, grounding, workloads as W

N_IN, N_OUT = 6, W.GROUND_SAMPLES


def generate(params, per_batch=512, log=None):
    """FDTD waveforms for every parameter row (shape [n, 6], the order of
    workloads.surrogate_inputs): domains are advanced per_batch at a time by
    the batched engine; the host builds the next batch while the GPU runs the
    current one (two streams).  Returns float32 waveforms [n, 512]."""
    import torch
    params = np.asarray(params, dtype=np.float64)
    n = len(params)
    out = np.empty((n, N_OUT), dtype=np.float32)
    steps = W.GROUND_STEPS
    block = grounding.tune_block(W.SURROGATE_N)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pending = None
    t0 = time.perf_counter()

    def finish(p):
        b, grids, lo = p
        b.synchronize()
        dt = grids[0].dt
        for i, g in enumerate(grids):
            out[lo + i] = W.impedance_waveform(g.read_probe(0, 0, steps), dt)
        b.close()
        for g in grids:
            g.close()

    for bi, lo in enumerate(range(0, n, per_batch)):
        s = streams[bi % 2]
        with torch.cuda.stream(s):
            grids = [fdtd.from_scenario(W.surrogate_domain(p), stream=s, probe_capacity=steps, block=block)
                     for p in params[lo:lo + per_batch]]
            b = fdtd.Batch(grids, stream=s)
            b.step(steps)
        if pending is not None:
            finish(pending)
        pending = (b, grids, lo)
        if log:
            log(f"batch {bi}: {min(lo + per_batch, n)}/{n} domains queued, {time.perf_counter() - t0:.1f} s")
    if pending is not None:
        finish(pending)
    return out


class Network:
    """A multilayer perceptron on the device: FP32 master weights with Adam
    moments, BF16 copies for the tensor cores, per-layer activation buffers
    for the backward pass.  sizes = [k0, n1, n2, ...]; acts[l] is the
    activation after layer l (mlp.ACT_GELU or mlp.ACT_NONE)."""

    def __init__(self, sizes, acts, seed=0, weights=None):
        import torch
        from . import mlp
        self.torch, self.mlp = torch, mlp
        self.sizes, self.acts = list(sizes), list(acts)
        rng = np.random.default_rng(seed)
        f32 = dict(dtype=torch.float32, device="cuda")
        self.W, self.b, self.Wb = [], [], []
        for l, (k, n) in enumerate(zip(sizes[:-1], sizes[1:])):
            if weights is not None:
                w0, b0 = weights[2 * l], weights[2 * l + 1]
            else:
                gain = np.sqrt(2.0) if acts[l] == mlp.ACT_GELU else 1.0
                w0, b0 = rng.standard_normal((n, k)) * gain / np.sqrt(k), np.zeros(n)
            self.W.append(torch.tensor(np.asarray(w0, np.float32), **f32).contiguous())
            self.b.append(torch.tensor(np.asarray(b0, np.float32), **f32).contiguous())
            self.Wb.append(torch.empty((n, k), dtype=torch.bfloat16, device="cuda"))
            mlp.to_bf16(self.W[-1], self.Wb[-1])
        self.params = [p for pair in zip(self.W, self.b) for p in pair]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.g = [torch.zeros_like(p) for p in self.params]
        self.t = 0
        self._bufs = {}
        self._image, self._image_t = None, None     # packed weights of forward_fused, and their Adam step
        self._fused_out = {}

    def _buffers(self, rows):
        """activation and gradient buffers, one set per row count and kept
        for the network's lifetime (a captured graph of a forward pass keeps
        pointing at the set of its batch size)"""
        if rows not in self._bufs:
            torch = self.torch
            f32 = dict(dtype=torch.float32, device="cuda")
            self._bufs[rows] = dict(
                z=[torch.empty((rows, n), **f32) for n in self.sizes[1:]],
                hb=[torch.empty((rows, n), dtype=torch.bfloat16, device="cuda") for n in self.sizes[1:-1]],
                out=torch.empty((rows, self.sizes[-1]), **f32),
                dz=[torch.empty((rows, n), **f32) for n in self.sizes[1:]],
                dh=[torch.empty((rows, n), **f32) for n in self.sizes[1:-1]])
        b = self._bufs[rows]
        self.z, self.hb, self.out, self.dz, self.dh = b["z"], b["hb"], b["out"], b["dz"], b["dh"]

    def forward(self, x, keep=True):
        """x: [rows, k0] FP32 (rounded to BF16 on load).  Returns the FP32
        output buffer [rows, n_last] (reused by the next call).  keep: store
        the pre-activations the backward pass needs (not for inference)."""
        rows = x.shape[0]
        self._buffers(rows)
        self.x = x
        h = x
        L = len(self.W)
        for l in range(L):
            last = l == L - 1
            self.mlp.forward(h, self.Wb[l], self.b[l], self.acts[l], None if last else self.hb[l],
                             self.out if last else None, self.z[l] if keep else None)
            h = None if last else self.hb[l]
        return self.out

    def forward_fused(self, x, out_scale=1.0):
        """Inference: the whole network in one launch (mlp.net_forward), bit
        for bit the per-layer chain, the output times out_scale.  x: [rows,
        k0] FP32.  Returns an FP32 [rows, n_last] buffer kept per row count
        (overwritten by the next call).  The packed weight image is rebuilt
        when Adam has changed the weights since it was packed."""
        torch = self.torch
        if self._image_t != self.t:
            if self._image is None:
                self._image = torch.empty(self.mlp.net_pack_bytes(self.sizes), dtype=torch.uint8, device="cuda")
            self.mlp.net_pack(self.sizes, self.Wb, self._image)
            self._image_t = self.t
        rows = x.shape[0]
        if rows not in self._fused_out:
            self._fused_out[rows] = torch.empty((rows, self.sizes[-1]), dtype=torch.float32, device="cuda")
        y = self._fused_out[rows]
        self.mlp.net_forward(x, self.sizes, self.acts, self._image, self.b, y, out_scale)
        return y

    def backward(self, dy):
        """gradients of every parameter from dL/d(output) [rows, n_last]"""
        L = len(self.W)
        for l in range(L - 1, -1, -1):
            x = self.x if l == 0 else self.hb[l - 1]
            self.mlp.backward(x, self.z[l], dy, self.Wb[l], self.acts[l], self.dz[l], self.g[2 * l],
                              self.g[2 * l + 1], None if l == 0 else self.dh[l - 1])
            dy = None if l == 0 else self.dh[l - 1]

    def adam(self, lr, weight_decay=0.0):
        self.t += 1
        for i, p in enumerate(self.params):
            wb = self.Wb[i // 2] if i % 2 == 0 else None
            self.mlp.adam(p, self.m[i], self.v[i], self.g[i], wb, lr, self.t,
                          weight_decay=weight_decay if i % 2 == 0 else 0.0)

    def host_weights(self):
        return [p.cpu().numpy() for p in self.params]


# -- input encoding and the trained model ----------------------------------
Y_UNIT = 100.0                      # ohm; network outputs are waveforms in these units
MAIN_SIZES = [N_IN, 256, 256, 256, N_OUT]
HEAD_SIZES = [N_IN, 64, 64, 1]


def features(params):
    """Encode parameter rows [n, 6] (eps_r, log10 sigma, length m, radius m,
    depth m, rise s) for the network: length and depth are quantised to the
    cells the domain builder uses (the FDTD model sees only those), then every
    input is mapped affinely (radius logarithmically) onto about [-1, 1] over
    its sampled range."""
    p = np.asarray(params, dtype=np.float64).reshape(-1, N_IN)
    cells = np.array([W.grounding_cells(l, d) for l, d in p[:, [2, 4]]], dtype=np.float64).reshape(-1, 2)
    length, depth = cells[:, 0] * W.GROUND_DX, cells[:, 1] * W.GROUND_DX
    return np.stack([(p[:, 0] - 22.0) / 18.0,
                     (p[:, 1] + 2.5) / 1.5,
                     (length - 5.0) / 4.0,
                     (np.log(p[:, 3]) - np.log(0.008)) / 0.7,
                     (depth - 0.5) / 0.5,
                     (p[:, 5] - 0.3e-6) / 0.2e-6], axis=1).astype(np.float32)


# sampled ranges of the six inputs (workloads.surrogate_inputs); the rod
# length must also fit the 64-cell domain: L + depth <= 10 m and <= 9 m
RANGES = ((4.0, 40.0), (-4.0, -1.0), (1.0, 10.0), (0.004, 0.016), (0.0, 1.0), (0.1e-6, 0.5e-6))


def in_range(params):
    """rows whose parameters lie inside the ranges the network was trained
    on (others always go to FDTD)"""
    p = np.asarray(params, dtype=np.float64).reshape(-1, N_IN)
    ok = np.ones(len(p), dtype=bool)
    for c, (lo, hi) in enumerate(RANGES):
        ok &= (p[:, c] >= lo) & (p[:, c] <= hi)
    lmax = min(10.0, W.GROUND_DX * (W.SURROGATE_N - 28))
    ok &= p[:, 2] + p[:, 4] <= lmax
    return ok


def _cosine(lr0, it, total):
    return lr0 * 0.5 * (1.0 + np.cos(np.pi * min(it, total) / max(total, 1)))


def fit(net, F, T, row_weight, epochs, batch=256, lr=1e-3, weight_decay=0.0, seed=0, log=None):
    """Minibatch Adam on the device: loss = mean_r w_r ||net(F_r) - T_r||^2.
    F [n, k0], T [n, n_last], row_weight [n] are device FP32 tensors."""
    import torch
    from . import mlp
    n = F.shape[0]
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    rng = np.random.default_rng(seed)
    f32 = dict(dtype=torch.float32, device="cuda")
    xb, tb = torch.empty((batch, F.shape[1]), **f32), torch.empty((batch, T.shape[1]), **f32)
    wb, dy = torch.empty((batch, 1), **f32), torch.empty((batch, T.shape[1]), **f32)
    loss = torch.zeros(1, **f32)
    w2 = row_weight.reshape(-1, 1)
    it = 0
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n)[:steps_per_epoch * batch].astype(np.int32), device="cuda")
        loss.zero_()
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            mlp.gather_rows(F, idx, xb)
            mlp.gather_rows(T, idx, tb)
            mlp.gather_rows(w2, idx, wb)
            out = net.forward(xb)
            mlp.mse(out, tb, 1.0 / batch, dy, loss, wb)
            net.backward(dy)
            net.adam(_cosine(lr, it, total), weight_decay)
            it += 1
        if log and (ep % 10 == 9 or ep == epochs - 1):
            log(f"epoch {ep + 1}/{epochs}: mean loss {loss.item() / steps_per_epoch:.3e}")
    return net


class Surrogate:
    """The trained waveform network plus its error head and acceptance
    threshold.  predict() runs both networks on the device;
    predict_with_fallback() re-runs rejected inputs through the FDTD
    engine."""

    def __init__(self, main, head, threshold, meta=None):
        self.main, self.head, self.threshold = main, head, float(threshold)
        self.meta = dict(meta or {})
        self._graphs = {}
        self._graphs_t = None           # the networks' Adam steps when the graphs were captured

    # -- inference ---------------------------------------------------------
    def predict_device(self, f_dev):
        """f_dev: encoded features [B, 6] on the device.  Returns device
        tensors (waveforms [B, 512] in ohm, predicted relative error [B]):
        each network in one launch, the waveform scaled to ohm in its
        output layer."""
        wave = self.main.forward_fused(f_dev, out_scale=Y_UNIT)
        log_err = self.head.forward_fused(f_dev)
        return wave, log_err.reshape(-1)

    def predict_graph(self, batch):
        """A CUDA graph of predict_device for `batch` rows, captured once per
        batch size: returns (input buffer [batch, 6], replay, outputs).  Copy
        encoded features into the input buffer, call replay(), read the
        outputs (device tensors, overwritten by the next replay)."""
        import torch
        if self._graphs_t != (self.main.t, self.head.t):
            # weights changed since the capture: the graphs would replay the
            # packed images of the old ones
            self._graphs = {}
            self._graphs_t = (self.main.t, self.head.t)
        if batch not in self._graphs:
            x = torch.zeros((batch, N_IN), dtype=torch.float32, device="cuda")
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                self.predict_device(x)          # allocates the layer buffers outside the capture
            torch.cuda.current_stream().wait_stream(side)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                wave, log_err = self.predict_device(x)
            self._graphs[batch] = (x, g, (wave, log_err))
        x, g, outs = self._graphs[batch]
        return x, g.replay, outs

    def predict(self, params):
        """waveforms [B, 512] (ohm) and the error head's predicted relative
        L2 error [B] for parameter rows [B, 6] (host arrays)."""
        f = features(params)
        x, replay, (wave, log_err) = self.predict_graph(len(f))
        x.copy_(__import__("torch").from_numpy(f), non_blocking=False)
        replay()
        return wave.cpu().numpy(), np.exp(log_err.cpu().numpy())

    def predict_with_fallback(self, params, max_err=None, per_batch=512):
        """Surrogate waveforms where the input lies in the trained ranges and
        the predicted error is within the acceptance threshold, FDTD
        waveforms elsewhere.  Returns (waveforms, accepted mask)."""
        thr = self.threshold if max_err is None else max_err
        wave, err = self.predict(params)
        acc = (err <= thr) & in_range(params)
        if (~acc).any():
            wave[~acc] = generate(np.asarray(params)[~acc], per_batch=per_batch)
        return wave, acc

    # -- persistence -------------------------------------------------------
    def save(self, path):
        import torch
        arrs = {}
        for name, net in (("main", self.main), ("head", self.head)):
            for l, (Wt, b) in enumerate(zip(net.W, net.b)):
                bits = Wt.to(torch.bfloat16).view(torch.int16).cpu().numpy().view(np.uint16)
                arrs[f"{name}_w{l}_bf16"] = bits
                arrs[f"{name}_b{l}"] = b.cpu().numpy()
        np.savez(path, threshold=np.float64(self.threshold), y_unit=np.float64(Y_UNIT),
                 main_sizes=np.array(MAIN_SIZES), head_sizes=np.array(HEAD_SIZES),
                 meta=np.array(repr(self.meta)), **arrs)

    @staticmethod
    def load(path):
        from . import mlp
        z = np.load(path)
        if float(z["y_unit"]) != Y_UNIT:
            raise ValueError("weight file uses a different output unit")

        def net(name, sizes):
            L = len(sizes) - 1
            ws = []
            for l in range(L):
                bits = z[f"{name}_w{l}_bf16"].astype(np.uint32) << 16
                ws += [bits.view(np.float32), z[f"{name}_b{l}"]]
            return Network(sizes, [mlp.ACT_GELU] * (L - 1) + [mlp.ACT_NONE], weights=ws)

        import ast
        return Surrogate(net("main", list(z["main_sizes"])), net("head", list(z["head_sizes"])),
                         float(z["threshold"]), ast.literal_eval(str(z["meta"])))


def train_surrogate(X, Y, n_cal, epochs=1600, head_epochs=600, target_err=0.02, max_exceed=0.01, seed=0,
                    log=None):
    """Train the waveform network on the first len(X) - n_cal rows and the
    error head on the network's log relative errors over the last n_cal rows
    (runs it has not seen).  The acceptance threshold is the largest
    predicted error for which, on the second half of the calibration rows
    (not used to fit the head), no more than a fraction max_exceed of the
    accepted runs exceed target_err."""
    import torch
    from . import mlp
    X = np.asarray(X)
    n_tr = len(X) - n_cal
    f32 = dict(dtype=torch.float32, device="cuda")
    F = torch.tensor(features(X), **f32)
    Tn = (np.asarray(Y, np.float64) / Y_UNIT).astype(np.float32)
    T = torch.tensor(Tn, **f32)
    w = torch.tensor((1.0 / np.sum(Tn.astype(np.float64) ** 2, axis=1)).astype(np.float32), **f32)
    gelu, none = mlp.ACT_GELU, mlp.ACT_NONE
    main = Network(MAIN_SIZES, [gelu, gelu, gelu, none], seed=seed)
    fit(main, F[:n_tr], T[:n_tr], w[:n_tr], epochs, seed=seed, log=log)
    # relative errors of the trained network on every row
    err = torch.empty(len(X), **f32)
    for lo in range(0, len(X), 4096):
        out = main.forward(F[lo:lo + 4096])
        mlp.row_rel_err(out, T[lo:lo + 4096], err[lo:lo + 4096])
    err_h = err.cpu().numpy().astype(np.float64)
    n_fit = n_cal // 2
    cal_fit = slice(n_tr, n_tr + n_fit)
    cal_thr = slice(n_tr + n_fit, len(X))
    le = torch.tensor(np.log(np.maximum(err_h, 1e-6)).astype(np.float32).reshape(-1, 1), **f32)
    head = Network(HEAD_SIZES, [gelu, gelu, none], seed=seed + 1)
    fit(head, F[cal_fit], le[cal_fit], torch.ones(n_fit, **f32), head_epochs, batch=128, lr=1e-3,
        seed=seed + 1, log=log)
    pe = np.empty(len(X))
    for lo in range(0, len(X), 4096):
        pe[lo:lo + 4096] = np.exp(head.forward(F[lo:lo + 4096]).cpu().numpy()[:, 0])
    thr = 0.0
    for cand in np.sort(pe[cal_thr]):
        acc = pe[cal_thr] <= cand
        if np.mean(err_h[cal_thr][acc] > target_err) <= max_exceed:
            thr = float(cand)
    meta = dict(n_train=n_tr, n_cal=n_cal, epochs=epochs, head_epochs=head_epochs, seed=seed,
                train_err_median=float(np.median(err_h[:n_tr])),
                cal_err_median=float(np.median(err_h[n_tr:])), target_err=target_err, max_exceed=max_exceed)
    return Surrogate(main, head, thr, meta), err_h, pe


# -- training entry point ----------------------------------------------------
TRAIN_SEEDS = (1, 20000)            # the last N_CAL of them calibrate the error head
HELDOUT_SEEDS = (20001, 22000)
N_CAL = 2000
WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__file__), "surrogate_weights.npz")


def dataset(lo, hi, cache=None, log=None):
    """(params [n, 6], FDTD waveforms [n, 512]) for seeds lo..hi, read from
    the npz cache when it holds exactly those seeds, else generated."""
    import os
    seeds = np.arange(lo, hi + 1)
    if cache and os.path.exists(cache):
        z = np.load(cache)
        sel = np.isin(z["seeds"], seeds)
        if sel.sum() == len(seeds):
            order = np.argsort(z["seeds"][sel])
            return z["X"][sel][order], z["Y"][sel][order]
    X = np.stack([W.surrogate_inputs(int(s)) for s in seeds])
    Y = generate(X, log=log)
    return X, Y


def nearest_neighbour_error(X_train, Y_train, X, Y):
    """The method without the network, as a baseline: answer each input with
    the FDTD waveform of the nearest training input (Euclidean distance of
    the encoded features).  Returns the relative L2 error per row (host
    evaluation of a baseline; not part of the surrogate)."""
    Ft, F = features(X_train).astype(np.float64), features(X).astype(np.float64)
    err = np.empty(len(F))
    for lo in range(0, len(F), 256):
        d2 = ((F[lo:lo + 256, None, :] - Ft[None, :, :]) ** 2).sum(-1)
        nn = np.argmin(d2, axis=1)
        y = np.asarray(Y[lo:lo + 256], np.float64)
        err[lo:lo + 256] = np.linalg.norm(np.asarray(Y_train, np.float64)[nn] - y, axis=1) / np.linalg.norm(y, axis=1)
    return err


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="generate the grounding dataset with the batched FDTD engine, "
                                             "train the surrogate on the GPU and evaluate it on held-out runs")
    ap.add_argument("--data", default=None, help="npz cache of (seeds, X, Y); written when generated")
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--report", default=None, help="JSON summary of training and held-out errors")
    ap.add_argument("--epochs", type=int, default=1600)
    ap.add_argument("--head-epochs", type=int, default=600)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)
    t0 = time.perf_counter()
    Xt, Yt = dataset(*TRAIN_SEEDS, cache=a.data, log=log)
    Xh, Yh = dataset(*HELDOUT_SEEDS, cache=a.data, log=log)
    t1 = time.perf_counter()
    if a.data and not __import__("os").path.exists(a.data):
        np.savez(a.data, seeds=np.arange(TRAIN_SEEDS[0], HELDOUT_SEEDS[1] + 1), X=np.concatenate([Xt, Xh]),
                 Y=np.concatenate([Yt, Yh]))
    sur, _, _ = train_surrogate(Xt, Yt, N_CAL, epochs=a.epochs, head_epochs=a.head_epochs, seed=a.seed, log=log)
    t2 = time.perf_counter()
    wave, err = sur.predict(Xh)
    rel = np.linalg.norm(wave - Yh, axis=1) / np.linalg.norm(Yh, axis=1)
    acc = (err <= sur.threshold) & in_range(Xh)
    nn = nearest_neighbour_error(Xt[:len(Xt) - N_CAL], Yt[:len(Xt) - N_CAL], Xh, Yh)
    rep = dict(data_s=t1 - t0, train_s=t2 - t1, threshold=sur.threshold,
               nearest_neighbour=dict(median=float(np.median(nn)), mean=float(nn.mean()),
                                      p99=float(np.percentile(nn, 99)), frac_le_2pct=float(np.mean(nn <= 0.02))),
               heldout=dict(
        n=len(Xh), median=float(np.median(rel)), mean=float(rel.mean()), p99=float(np.percentile(rel, 99)),
        max=float(rel.max()), frac_le_2pct=float(np.mean(rel <= 0.02)), accepted=float(acc.mean()),
        max_accepted=float(rel[acc].max()) if acc.any() else None), **sur.meta)
    sur.meta.update(heldout=rep["heldout"])
    sur.save(a.out)
    log(json.dumps(rep))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
