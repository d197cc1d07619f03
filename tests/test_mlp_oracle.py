"""Pins of the FP64 network oracle (CPU): GELU closed-form values, the
backward pass against central finite differences, the first Adam step's
closed form, and BF16 rounding against its definition."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M


def test_gelu_values():
    # z Phi(z): Phi(0) = 1/2, Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457
    assert M.gelu(np.array(0.0)) == 0.0
    assert abs(M.gelu(np.array(1.0)) - 0.841344746068543) < 1e-14
    assert abs(M.gelu(np.array(-1.0)) + 0.158655253931457) < 1e-14
    assert abs(M.gelu_grad(np.array(0.0)) - 0.5) < 1e-15
    z = np.linspace(-4, 4, 81)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.gelu_grad(z))) < 1e-8


def make_net(rng, sizes):
    layers = []
    for k, n in zip(sizes[:-1], sizes[1:]):
        layers.append((rng.standard_normal((n, k)) / math.sqrt(k), rng.standard_normal(n) * 0.1))
    acts = ["gelu"] * (len(sizes) - 2) + ["none"]
    return layers, acts


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    layers, acts = make_net(rng, [6, 9, 7, 5])
    x = rng.standard_normal((11, 6))
    t = rng.standard_normal((11, 5))

    def loss(ls, xx):
        return M.mse(M.forward(xx, ls, acts)[2], t, 1.0 / t.size)[0]

    _, _, y = M.forward(x, layers, acts)
    _, dout = M.mse(y, t, 1.0 / t.size)
    grads, dx = M.backward(x, layers, acts, dout)
    h = 1e-6
    for l, (W, b) in enumerate(layers):
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2 % W.shape[1])]:
            Wp = [(w.copy(), bb.copy()) for w, bb in layers]
            Wm = [(w.copy(), bb.copy()) for w, bb in layers]
            Wp[l][0][i, j] += h
            Wm[l][0][i, j] -= h
            fd = (loss(Wp, x) - loss(Wm, x)) / (2 * h)
            assert abs(fd - grads[l][0][i, j]) < 1e-7 * max(1.0, abs(fd))
        bp = [(w.copy(), bb.copy()) for w, bb in layers]
        bm = [(w.copy(), bb.copy()) for w, bb in layers]
        bp[l][1][0] += h
        bm[l][1][0] -= h
        assert abs((loss(bp, x) - loss(bm, x)) / (2 * h) - grads[l][1][0]) < 1e-7
    xp, xm = x.copy(), x.copy()
    xp[3, 2] += h
    xm[3, 2] -= h
    assert abs((loss(layers, xp) - loss(layers, xm)) / (2 * h) - dx[3, 2]) < 1e-7


def test_adam_first_step_is_signed_lr():
    """with m = v = 0, t = 1 and eps -> 0 the first step is -lr sign(g)"""
    g = np.array([0.3, -2.0, 1e-3])
    w, m, v = M.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 0.01, 0.9, 0.999, 1e-15, 0.0, 1)
    np.testing.assert_allclose(w, -0.01 * np.sign(g), rtol=1e-9)


def test_bf16_rounding():
    # exactly representable values survive; 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even (1)
    assert M.bf16(np.array(1.5)) == 1.5
    assert M.bf16(np.array(1.0 + 2.0 ** -8)) == 1.0
    assert M.bf16(np.array(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6
    x = np.random.default_rng(1).standard_normal(1000)
    assert np.max(np.abs(M.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_weighted_mse_is_sum_of_squared_relative_errors():
    """with w_r = 1/||t_r||^2 the weighted loss is sum_r (||y_r - t_r|| / ||t_r||)^2;
    its gradient matches central differences"""
    rng = np.random.default_rng(4)
    y, t = rng.standard_normal((5, 9)), rng.standard_normal((5, 9)) * 3
    w = 1.0 / np.sum(t * t, axis=1)
    loss, dy = M.mse(y, t, 0.5, w)
    rel = np.linalg.norm(y - t, axis=1) / np.linalg.norm(t, axis=1)
    assert loss == pytest.approx(0.5 * np.sum(rel ** 2), rel=1e-12)
    h = 1e-6
    for r, c in [(0, 0), (2, 5), (4, 8)]:
        yp, ym = y.copy(), y.copy()
        yp[r, c] += h
        ym[r, c] -= h
        fd = (M.mse(yp, t, 0.5, w)[0] - M.mse(ym, t, 0.5, w)[0]) / (2 * h)
        assert dy[r, c] == pytest.approx(fd, rel=1e-7)


def test_adam_bias_corrections_hold_at_every_step():
    """with a constant gradient the bias-corrected moments are g and g^2 at
    every step t, so each step is exactly -lr sign(g) (eps -> 0): after T
    steps w = -T lr sign(g)"""
    g = np.array([0.7, -1.3, 2e-3])
    w, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 26):
        w, m, v = M.adam(w, m, v, g, 0.01, 0.9, 0.999, 1e-15, 0.0, t)
    np.testing.assert_allclose(w, -25 * 0.01 * np.sign(g), rtol=1e-9)


def test_adam_weight_decay_is_decoupled():
    """with zero gradients the moments stay zero and decoupled weight decay
    alone acts: w_t = w_0 (1 - lr wd)^t"""
    w0 = np.array([1.0, -2.0, 0.5])
    w, m, v = w0.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 11):
        w, m, v = M.adam(w, m, v, np.zeros(3), 0.01, 0.9, 0.999, 1e-8, 0.1, t)
    np.testing.assert_allclose(w, w0 * (1 - 0.01 * 0.1) ** 10, rtol=1e-12)
