"""Host-side parts of the surrogate: input encoding, trained-range check and
the committed weight file's layout (no GPU)."""
import os

import numpy as np

from paper_2207_06908_gb300 import surrogate as S, workloads as W


def test_features_quantise_like_the_domain_builder():
    X = np.stack([W.surrogate_inputs(s) for s in range(1, 400)])
    F = S.features(X)
    assert F.shape == (len(X), 6) and F.dtype == np.float32
    assert np.all(np.abs(F) <= 1.0 + 1e-6)
    for x, f in zip(X[:50], F[:50]):
        lc, dc = W.grounding_cells(x[2], x[4])
        sc = W.surrogate_domain(x)
        rod = sc.wires[0]
        assert rod[1][2] - rod[0][2] == lc                      # rod length in cells
        assert (sc.n[2] - 14) - rod[1][2] == dc                 # rod top below the surface
        assert np.isclose(f[2], (lc * W.GROUND_DX - 5.0) / 4.0, atol=1e-6)
        assert np.isclose(f[4], (dc * W.GROUND_DX - 0.5) / 0.5, atol=1e-6)
    # inputs that round to the same cells encode identically in length and depth
    a, b = X[0].copy(), X[0].copy()
    b[2] = a[2] + 0.01 if round((a[2] + 0.01) / 0.25) == round(a[2] / 0.25) else a[2] - 0.01
    assert S.features(a)[0, 2] == S.features(b)[0, 2]


def test_in_range():
    X = np.stack([W.surrogate_inputs(s) for s in range(1, 200)])
    assert S.in_range(X).all()
    for c, v in [(0, 3.9), (0, 41.0), (1, -4.2), (1, -0.9), (3, 0.02), (5, 0.6e-6)]:
        y = X[:1].copy()
        y[0, c] = v
        assert not S.in_range(y)[0]
    y = X[:1].copy()
    y[0, 2], y[0, 4] = 8.6, 0.6          # rod does not fit the 64-cell domain
    assert not S.in_range(y)[0]


def test_weight_file_layout():
    assert os.path.exists(S.WEIGHTS), "trained weights are part of the package"
    z = np.load(S.WEIGHTS)
    assert list(z["main_sizes"]) == S.MAIN_SIZES and list(z["head_sizes"]) == S.HEAD_SIZES
    for name, sizes in (("main", S.MAIN_SIZES), ("head", S.HEAD_SIZES)):
        for l, (k, n) in enumerate(zip(sizes[:-1], sizes[1:])):
            assert z[f"{name}_w{l}_bf16"].shape == (n, k) and z[f"{name}_w{l}_bf16"].dtype == np.uint16
            assert z[f"{name}_b{l}"].shape == (n,)
    assert 0.0 < float(z["threshold"]) <= 0.05
    assert float(z["y_unit"]) == S.Y_UNIT
