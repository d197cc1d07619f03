"""Surrogate-network kernels (BF16 operands, FP32 accumulation, tcgen05
tensor cores for every contraction) against the FP64 oracle on the same
BF16-rounded weights and inputs.
FP32 outputs of exact BF16 products: 1e-4 relative L2; outputs that pass
through BF16 (stored activations, dz entering the weight / input gradient
GEMMs): 1e-2."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import mlp
    return torch, mlp


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(torch, a, dtype):
    return torch.tensor(np.asarray(a, np.float32), device="cuda").to(dtype).contiguous()


@pytest.mark.parametrize("rows,k,n,act", [(300, 70, 130, 1), (64, 256, 256, 1), (4096, 6, 256, 1),
                                          (257, 256, 512, 0), (1, 13, 7, 1), (129, 64, 1, 0), (200, 300, 40, 1),
                                          (131, 24, 200, 1)])
def test_forward_layer(env, rows, k, n, act):
    torch, mlp = env
    rng = np.random.default_rng(rows + k + n)
    x = M.bf16(rng.standard_normal((rows, k)))
    W = M.bf16(rng.standard_normal((n, k)) / np.sqrt(k))
    b = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    xd, Wd, bd = dev(torch, x, torch.bfloat16), dev(torch, W, torch.bfloat16), dev(torch, b, torch.float32)
    yb = torch.empty((rows, n), dtype=torch.bfloat16, device="cuda")
    yf = torch.empty((rows, n), dtype=torch.float32, device="cuda")
    zf = torch.empty((rows, n), dtype=torch.float32, device="cuda")
    mlp.forward(xd, Wd, bd, act, yb, yf, zf)
    mlp.check()
    _, zs, y = M.forward(x, [(W, b)], ["gelu" if act else "none"])
    assert rel(zf.cpu().numpy(), zs[0]) <= 1e-4
    assert rel(yf.cpu().numpy(), y) <= 1e-4
    assert rel(yb.float().cpu().numpy(), y) <= 1e-2


@pytest.mark.parametrize("rows,k,n,act", [(300, 70, 130, 1), (512, 256, 512, 0), (77, 6, 256, 1),
                                          (1000, 256, 256, 1), (9, 33, 3, 0)])
def test_backward_layer(env, rows, k, n, act):
    torch, mlp = env
    rng = np.random.default_rng(3 * rows + k)
    x = M.bf16(rng.standard_normal((rows, k)))
    W = M.bf16(rng.standard_normal((n, k)) / np.sqrt(k))
    b = np.zeros(n)
    dy = rng.standard_normal((rows, n)).astype(np.float32).astype(np.float64)
    _, zs, _ = M.forward(x, [(W, b)], ["gelu" if act else "none"])
    z32 = zs[0].astype(np.float32).astype(np.float64)
    dz, dW, db, dx = M.layer_backward(x, z32, dy, W, "gelu" if act else "none")
    xd, Wd = dev(torch, x, torch.bfloat16), dev(torch, W, torch.bfloat16)
    zd, dyd = dev(torch, z32, torch.float32), dev(torch, dy, torch.float32)
    f32 = dict(dtype=torch.float32, device="cuda")
    dzd, dwd, dbd, dxd = (torch.empty((rows, n), **f32), torch.empty((n, k), **f32), torch.empty(n, **f32),
                          torch.empty((rows, k), **f32))
    mlp.backward(xd, zd, dyd, Wd, act, dzd, dwd, dbd, dxd)
    torch.cuda.synchronize()
    assert rel(dzd.cpu().numpy(), dz) <= 1e-5
    assert rel(dbd.cpu().numpy(), db) <= 1e-5
    assert rel(dwd.cpu().numpy(), dW) <= 1e-2
    assert rel(dxd.cpu().numpy(), dx) <= 1e-2


def test_network_gradients_vs_oracle(env):
    """6 -> 256 -> 256 -> 256 -> 512 with GELU, MSE loss: every weight and
    bias gradient of the GPU chain within 1e-2 of the FP64 oracle"""
    torch, mlp = env
    rng = np.random.default_rng(11)
    sizes = [6, 256, 256, 256, 512]
    layers = [(M.bf16(rng.standard_normal((n, k)) / np.sqrt(k)), rng.standard_normal(n) * 0.05)
              for k, n in zip(sizes[:-1], sizes[1:])]
    layers = [(W, b.astype(np.float32).astype(np.float64)) for W, b in layers]
    acts = ["gelu", "gelu", "gelu", "none"]
    rows = 192
    x = M.bf16(rng.uniform(-1, 1, (rows, 6)))
    t = rng.standard_normal((rows, 512)) * 0.5
    scale = 1.0 / t.size
    f32 = dict(dtype=torch.float32, device="cuda")
    h = dev(torch, x, torch.bfloat16)
    ins, zs, Wds = [h], [], []
    for l, ((W, b), act) in enumerate(zip(layers, acts)):
        n = W.shape[0]
        Wd = dev(torch, W, torch.bfloat16)
        Wds.append(Wd)
        z = torch.empty((rows, n), **f32)
        yb = torch.empty((rows, n), dtype=torch.bfloat16, device="cuda")
        yf = torch.empty((rows, n), **f32)
        mlp.forward(ins[-1], Wd, dev(torch, b, torch.float32), 1 if act == "gelu" else 0, yb, yf, z)
        zs.append(z)
        ins.append(yb if l < len(layers) - 1 else yf)
    loss = torch.zeros(1, **f32)
    dy = torch.empty((rows, 512), **f32)
    rw = 1.0 / np.sum(t.astype(np.float32).astype(np.float64) ** 2, axis=1)
    mlp.mse(ins[-1], dev(torch, t, torch.float32), scale, dy, loss, dev(torch, rw, torch.float32))
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        n, k = layers[l][0].shape
        dz = torch.empty((rows, n), **f32)
        dw, db = torch.empty((n, k), **f32), torch.empty(n, **f32)
        dx = torch.empty((rows, k), **f32) if l > 0 else None
        mlp.backward(ins[l], zs[l], dy, Wds[l], 1 if acts[l] == "gelu" else 0, dz, dw, db, dx)
        grads[l] = (dw, db)
        dy = dx
    torch.cuda.synchronize()
    _, _, yo = M.forward(x, layers, acts)
    lo, dout = M.mse(yo, t, scale, rw)
    ref, _ = M.backward(x, layers, acts, dout)
    assert abs(loss.item() - lo) <= 1e-2 * lo
    for l in range(len(layers)):
        assert rel(grads[l][0].cpu().numpy(), ref[l][0]) <= 1e-2, l
        assert rel(grads[l][1].cpu().numpy(), ref[l][1]) <= 1e-2, l


def test_adam_step(env):
    torch, mlp = env
    rng = np.random.default_rng(5)
    n = 10007
    w, m, v, g = (rng.standard_normal(n) for _ in range(4))
    v = np.abs(v)
    f = lambda a: dev(torch, a, torch.float32)
    wd_, md, vd, gd = f(w), f(m), f(v), f(g)
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    mlp.adam(wd_, md, vd, gd, wb, 1e-3, 7, weight_decay=1e-4)
    torch.cuda.synchronize()
    w32, m32, v32, g32 = (a.astype(np.float32).astype(np.float64) for a in (w, m, v, g))
    wr, mr, vr = M.adam(w32, m32, v32, g32, 1e-3, 0.9, 0.999, 1e-8, 1e-4, 7)
    assert rel(wd_.cpu().numpy(), wr) <= 1e-6
    assert rel(md.cpu().numpy(), mr) <= 1e-6
    assert rel(vd.cpu().numpy(), vr) <= 1e-6
    np.testing.assert_array_equal(wb.float().cpu().numpy(), M.bf16(wd_.cpu().numpy()).astype(np.float32))


def test_row_kernels(env):
    """weighted squared error, per-row relative error, row gather and row
    scaling on a ragged shape"""
    torch, mlp = env
    rng = np.random.default_rng(8)
    rows, cols = 37, 515
    y = rng.standard_normal((rows, cols)).astype(np.float32).astype(np.float64)
    t = rng.standard_normal((rows, cols)).astype(np.float32).astype(np.float64)
    t[3] = 0.0
    w = rng.uniform(0.5, 2.0, rows).astype(np.float32).astype(np.float64)
    f32 = dict(dtype=torch.float32, device="cuda")
    yd, td, wd = dev(torch, y, torch.float32), dev(torch, t, torch.float32), dev(torch, w, torch.float32)
    loss, dy, err = torch.zeros(1, **f32), torch.empty((rows, cols), **f32), torch.empty(rows, **f32)
    mlp.mse(yd, td, 0.25, dy, loss, wd)
    mlp.row_rel_err(yd, td, err)
    idx = rng.integers(0, rows, 50).astype(np.int32)
    g = torch.empty((50, cols), **f32)
    mlp.gather_rows(yd, torch.tensor(idx, device="cuda"), g)
    s = rng.uniform(-3, 3, rows)
    ys = yd.clone()
    mlp.scale_rows(ys, dev(torch, s, torch.float32))
    torch.cuda.synchronize()
    lo, dref = M.mse(y, t, 0.25, w)
    assert loss.item() == pytest.approx(lo, rel=1e-5)
    assert rel(dy.cpu().numpy(), dref) <= 1e-6
    e = np.linalg.norm(y - t, axis=1)
    nt = np.linalg.norm(t, axis=1)
    ref = np.where(nt > 0, e / np.where(nt > 0, nt, 1), e)
    np.testing.assert_allclose(err.cpu().numpy(), ref, rtol=1e-5)
    np.testing.assert_array_equal(g.cpu().numpy(), y[idx].astype(np.float32))
    assert rel(ys.cpu().numpy(), y * s.astype(np.float32)[:, None]) <= 1e-7


def test_forward_layer_fp32_input(env):
    """FP32 inputs are rounded to BF16 on load (the first surrogate layer)"""
    torch, mlp = env
    rng = np.random.default_rng(77)
    rows, k, n = 515, 6, 256
    x = rng.uniform(-1, 1, (rows, k)).astype(np.float32).astype(np.float64)
    W = M.bf16(rng.standard_normal((n, k)) / np.sqrt(k))
    b = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    yf = torch.empty((rows, n), dtype=torch.float32, device="cuda")
    mlp.forward(dev(torch, x, torch.float32), dev(torch, W, torch.bfloat16), dev(torch, b, torch.float32), 1,
                None, yf, None)
    mlp.check()
    _, _, y = M.forward(M.bf16(x), [(W, b)], ["gelu"])
    assert rel(yf.cpu().numpy(), y) <= 1e-4


def _layer_chain(torch, mlp, x, Wd, bd, acts, out_scale):
    """the per-layer path: BF16 hidden activations, FP32 output, then scaled"""
    h = x
    for l, (w, b) in enumerate(zip(Wd, bd)):
        n = w.shape[0]
        if l < len(Wd) - 1:
            nxt = torch.empty((x.shape[0], n), dtype=torch.bfloat16, device="cuda")
            mlp.forward(h, w, b, acts[l], nxt, None, None)
            h = nxt
        else:
            y = torch.empty((x.shape[0], n), dtype=torch.float32, device="cuda")
            mlp.forward(h, w, b, acts[l], None, y, None)
    return (y.cpu().numpy() * np.float32(out_scale)).astype(np.float32)


@pytest.mark.parametrize("sizes,acts,rows,scale", [
    ([6, 256, 256, 256, 512], [1, 1, 1, 0], 4096, 1000.0),   # the waveform network at the benchmark's batch
    ([6, 256, 256, 256, 512], [1, 1, 1, 0], 300, 1.0),       # ragged last row tile
    ([6, 64, 64, 1], [1, 1, 0], 129, 1.0),                   # the error head (one output column)
    ([13, 100, 37, 5], [0, 1, 1], 1, 0.5),                   # unaligned widths, a linear hidden layer
    ([256, 256], [1], 257, 1.0),                             # one layer, the largest K
    ([24, 48, 200, 96, 64, 32, 16], [1, 1, 1, 1, 1, 0], 520, 2.0),   # six layers
])
def test_fused_network_matches_layer_chain(env, sizes, acts, rows, scale):
    """The whole network in one clustered launch equals, bit for bit, the
    chain of per-layer launches (same BF16 roundings and K steps), and the
    FP64 network oracle within the BF16-activation bar"""
    torch, mlp = env
    rng = np.random.default_rng(sum(sizes) + rows)
    x = rng.standard_normal((rows, sizes[0])).astype(np.float32)
    Ws = [M.bf16(rng.standard_normal((n, k)) / np.sqrt(k)) for k, n in zip(sizes[:-1], sizes[1:])]
    bs = [rng.standard_normal(n).astype(np.float32).astype(np.float64) * 0.1 for n in sizes[1:]]
    xd = torch.tensor(x, device="cuda")
    Wd = [dev(torch, w, torch.bfloat16) for w in Ws]
    bd = [dev(torch, b, torch.float32) for b in bs]
    image = torch.empty(mlp.net_pack_bytes(sizes), dtype=torch.uint8, device="cuda")
    mlp.net_pack(sizes, Wd, image)
    y = torch.empty((rows, sizes[-1]), dtype=torch.float32, device="cuda")
    mlp.net_forward(xd, sizes, acts, image, bd, y, scale)
    mlp.check()
    got = y.cpu().numpy()
    want = _layer_chain(torch, mlp, xd, Wd, bd, acts, scale)
    mlp.check()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), np.abs(got - want).max()
    names = ["gelu" if a else "none" for a in acts]
    ref = M.forward(M.bf16(x.astype(np.float64)), list(zip(Ws, bs)), names)[2] * scale
    assert rel(got, ref) <= 1e-2


def test_fused_network_twice_and_without_bias(env):
    """back-to-back launches on one image give the same outputs; a null bias
    entry is no bias"""
    torch, mlp = env
    sizes, acts = [6, 64, 64, 8], [1, 1, 0]
    rng = np.random.default_rng(9)
    x = torch.tensor(rng.standard_normal((200, 6)).astype(np.float32), device="cuda")
    Wd = [dev(torch, M.bf16(rng.standard_normal((n, k)) / np.sqrt(k)), torch.bfloat16)
          for k, n in zip(sizes[:-1], sizes[1:])]
    zero = [torch.zeros(n, dtype=torch.float32, device="cuda") for n in sizes[1:]]
    image = torch.empty(mlp.net_pack_bytes(sizes), dtype=torch.uint8, device="cuda")
    mlp.net_pack(sizes, Wd, image)
    ys = []
    for biases in ([None, None, None], zero, [None, zero[1], None]):
        y = torch.empty((200, 8), dtype=torch.float32, device="cuda")
        mlp.net_forward(x, sizes, acts, image, biases, y)
        ys.append(y.cpu().numpy())
    mlp.check()
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])
