"""The learned surrogate against the FDTD engine it replaces (GPU).

The committed network was trained by the library's own BF16 kernels on
FDTD runs of seeds 1..20000; these tests use held-out seeds only."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_06908_gb300 import surrogate as S, workloads as W
    return torch, S, W


def held_out(W, S, n, first=None):
    lo = S.HELDOUT_SEEDS[0] if first is None else first
    return np.stack([W.surrogate_inputs(s) for s in range(lo, lo + n)])


def test_surrogate_gain_over_fdtd(env):
    """On 256 held-out inputs: every accepted waveform within 2% relative L2
    of FDTD, and surrogate-plus-fallback throughput at least 100x the
    batched FDTD engine's on the same inputs"""
    torch, S, W = env
    sur = S.Surrogate.load(S.WEIGHTS)
    X = held_out(W, S, 256)
    t0 = time.perf_counter()
    Y = S.generate(X)
    s_fdtd = len(X) / (time.perf_counter() - t0)
    wave, perr = sur.predict(X)
    rel = np.linalg.norm(wave - Y, axis=1) / np.linalg.norm(Y, axis=1)
    acc = (perr <= sur.threshold) & S.in_range(X)
    assert acc.mean() >= 0.95
    assert rel[acc].max() <= 0.02
    assert np.median(rel) <= 0.01
    # inference throughput at batch 4096
    f = torch.tensor(S.features(held_out(W, S, 4096)), device="cuda")
    for _ in range(3):
        sur.predict_device(f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        sur.predict_device(f)
    torch.cuda.synchronize()
    s_sur = 20 * 4096 / (time.perf_counter() - t0)
    fb = 1.0 - acc.mean()
    combined = 1.0 / ((1 - fb) / s_sur + fb / s_fdtd)
    assert combined >= 100 * s_fdtd, (combined, s_fdtd)


def test_fallback_runs_fdtd_outside_trained_ranges(env):
    """inputs outside the sampled ranges are never answered by the network:
    their waveforms are the FDTD engine's, bit for bit"""
    torch, S, W = env
    sur = S.Surrogate.load(S.WEIGHTS)
    X = held_out(W, S, 4)
    X[1, 0] = 60.0          # eps_r above the trained range
    X[3, 1] = -0.5          # sigma above the trained range
    wave, acc = sur.predict_with_fallback(X)
    assert not acc[1] and not acc[3]
    Y = S.generate(X[[1, 3]])
    np.testing.assert_array_equal(wave[[1, 3]], Y)


def test_training_learns_fdtd_waveforms(env):
    """a fresh network trained by the library's kernels on 256 FDTD runs
    fits them far better than at initialisation and generalises to unseen
    runs of the same generator"""
    torch, S, W = env
    from paper_2207_06908_gb300 import mlp
    X = held_out(W, S, 320, first=40001)
    Y = S.generate(X)
    f32 = dict(dtype=torch.float32, device="cuda")
    F = torch.tensor(S.features(X), **f32)
    Tn = (Y / S.Y_UNIT).astype(np.float32)
    T = torch.tensor(Tn, **f32)
    w = torch.tensor(1.0 / np.sum(Tn.astype(np.float64) ** 2, axis=1), **f32)
    g = mlp.ACT_GELU
    net = S.Network(S.MAIN_SIZES, [g, g, g, mlp.ACT_NONE], seed=3)

    def err(lo, hi):
        e = torch.empty(hi - lo, **f32)
        mlp.row_rel_err(net.forward(F[lo:hi]), T[lo:hi], e)
        return float(np.median(e.cpu().numpy()))

    e0 = err(256, 320)
    S.fit(net, F[:256], T[:256], w[:256], epochs=400, batch=64, lr=1e-3)
    e_tr, e_ho = err(0, 256), err(256, 320)
    assert e_tr <= 0.05 and e_ho <= 0.1 and e_ho <= e0 / 5, (e0, e_tr, e_ho)


def test_full_batch_inference_matches_network_oracle(env):
    """The inference the benchmark times (batch 4096 replayed from the
    captured graph): on 64 sampled rows the waveform network and the error
    head agree with the FP64 network oracle on the same BF16 weights and
    BF16-rounded inputs within 1e-2 (relative L2)"""
    torch, S, W = env
    from oracle import mlp_oracle as M
    from paper_2207_06908_gb300 import mlp
    sur = S.Surrogate.load(S.WEIGHTS)
    B = 4096
    f = S.features(held_out(W, S, B))
    x, replay, (wave, log_err) = sur.predict_graph(B)
    x.copy_(torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)))
    replay()
    torch.cuda.synchronize()
    wave, log_err = wave.cpu().numpy(), log_err.cpu().numpy()
    rows = np.random.default_rng(5).choice(B, 64, replace=False)
    xin = M.bf16(np.asarray(f, np.float32)[rows].astype(np.float64))

    def reference(net):
        layers = [(Wb.float().cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64))
                  for Wb, b in zip(net.Wb, net.b)]
        acts = ["gelu" if a == mlp.ACT_GELU else "none" for a in net.acts]
        return M.forward(xin, layers, acts)[2]

    ref_wave = reference(sur.main) * S.Y_UNIT
    got = wave[rows].astype(np.float64)
    assert np.linalg.norm(got - ref_wave) / np.linalg.norm(ref_wave) <= 1e-2
    ref_err = reference(sur.head).reshape(-1)
    assert np.linalg.norm(log_err[rows] - ref_err) / np.linalg.norm(ref_err) <= 1e-2
