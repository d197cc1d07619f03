"""FP64 reference of the surrogate network (a multilayer perceptron with
GELU), used to check the BF16 tensor-core kernels of the library.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and bench.py's reference
legs); the CUDA library never imports it.  Plain numpy, FP64.

The network: layer l computes z = x W^T + b, y = act(z) with GELU
act(z) = z Phi(z) = 0.5 z (1 + erf(z / sqrt 2)) on hidden layers and the
identity on the last; the loss is the mean squared error; training uses
Adam (Kingma and Ba) with bias-corrected moments.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)"""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(x, layers, acts):
    """layers: [(W [n x k], b [n])]; acts: 'gelu' | 'none' per layer.
    Returns the per-layer inputs and pre-activations and the output."""
    xs, zs = [], []
    h = np.asarray(x, dtype=np.float64)
    for (W, b), act in zip(layers, acts):
        xs.append(h)
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        zs.append(z)
        h = gelu(z) if act == "gelu" else z
    return xs, zs, h


def layer_backward(x, z, dy, W, act):
    """one layer: dz = dy act'(z); dW = dz^T x; db = sum dz; dx = dz W"""
    dz = dy * gelu_grad(z) if act == "gelu" else dy
    return dz, dz.T @ x, dz.sum(axis=0), dz @ np.asarray(W, np.float64)


def backward(x, layers, acts, dout):
    xs, zs, _ = forward(x, layers, acts)
    grads = [None] * len(layers)
    d = np.asarray(dout, np.float64)
    for l in range(len(layers) - 1, -1, -1):
        _, dW, db, d = layer_backward(xs[l], zs[l], d, layers[l][0], acts[l])
        grads[l] = (dW, db)
    return grads, d


def mse(y, t, scale, row_weight=None):
    """scale * sum_r w_r ||y_r - t_r||^2 and its gradient with respect to y"""
    e = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    w = np.ones(e.shape[0]) if row_weight is None else np.asarray(row_weight, np.float64)
    return scale * float(np.sum(w[:, None] * e * e)), 2.0 * scale * w[:, None] * e


def adam(w, m, v, g, lr, b1, b2, eps, wd, t):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    w = w - lr * mh / (np.sqrt(vh) + eps) - lr * wd * w
    return w, m, v


def bf16(a):
    """round to the nearest bfloat16 (ties to even), returned as float64"""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
