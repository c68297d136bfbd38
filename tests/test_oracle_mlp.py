"""The FP64 oracle MLP's backpropagation against central finite differences,
and its bfloat16 rounding against the bit-level definition."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    w = rng.standard_normal(mlp.n_params()) * 0.05
    X = rng.standard_normal((5, 16))
    T = rng.standard_normal((5, 325))
    M = (rng.random((5, 325)) < 0.4).astype(float)
    L, g = mlp.loss_and_grad(w, X, T, M)
    assert abs(L - mlp.loss(w, X, T, M)) < 1e-14 * max(1.0, L)
    idx = rng.choice(w.size, size=60, replace=False)
    idx = np.concatenate([idx, [0, 4095, 4096, 4351, 4352, 4352 + 65535, w.size - 1]])
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss(wp, X, T, M) - mlp.loss(wm, X, T, M)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.1415926, 1e-30, 65504.0], dtype=np.float32)
    r = mlp.to_bf16(vals)
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2.0 ** -8)
    assert r[0] == 1.0 and r[1] == 1.0  # halfway case rounds to even
