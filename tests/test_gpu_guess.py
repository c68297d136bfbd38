"""Learned initial guess: the GPU MLP against the FP64 oracle MLP, the pair
features against their definition, and training + SCF behaviour."""
import numpy as np
import pytest

from paper_1708_00033_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_00033_gb300 import hf
    return hf.Context(0)


def _bf16_weights(w):
    """Weight matrices as the kernels use them (bf16), biases as stored (fp32)."""
    from oracle import mlp
    out = np.asarray(w, dtype=np.float64).copy()
    o = 0
    for s in mlp.SHAPES:
        k = int(np.prod(s))
        if len(s) == 2:
            out[o:o + k] = mlp.to_bf16(w[o:o + k])
        o += k
    return out


def test_forward_and_gradients_vs_oracle(ctx):
    import torch
    from oracle import mlp
    from paper_1708_00033_gb300 import guess, hf
    rng = np.random.default_rng(5)
    w0 = guess.init_weights(3)
    w0[-325:] = rng.standard_normal(325).astype(np.float32) * 0.1
    model = hf.Model(ctx, w0)
    n = 300
    X = rng.standard_normal((n, 16)).astype(np.float32)
    T = rng.standard_normal((n, 325)).astype(np.float32)
    M = np.zeros((n, 325), dtype=np.float32)
    heads = rng.integers(0, 3, n)
    for i, h in enumerate(heads):
        M[i, (0, 225, 300)[h]:(225, 300, 325)[h]] = 1.0
    wq = _bf16_weights(w0)
    Y_ref, _ = mlp.forward(wq, X)
    Y = model.forward(X)
    assert np.abs(Y - Y_ref).max() <= 2e-4 * np.abs(Y_ref).max()
    dev = torch.device("cuda")
    loss = model.train_step(torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev), torch.from_numpy(M).to(dev), 0.0)
    L_ref, g_ref = mlp.loss_and_grad(wq, X, T, M)
    assert abs(loss - L_ref) <= 1e-4 * L_ref
    g = model.weights(gradients=True)
    o = 0
    for s in mlp.SHAPES:
        k = int(np.prod(s))
        scale = np.abs(g_ref[o:o + k]).max()
        assert np.abs(g[o:o + k] - g_ref[o:o + k]).max() <= 1e-3 * scale, s
        o += k
    # one Adam step moves the weights along -grad
    model.train_step(torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev), torch.from_numpy(M).to(dev), 1e-3)
    dw = model.weights() - w0
    assert np.mean(np.sign(dw[np.abs(g_ref) > 1e-6]) == -np.sign(g_ref[np.abs(g_ref) > 1e-6])) > 0.99


def test_features_match_geometry(ctx):
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(2, 5, 1)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis)
    X, meta = hf.guess_features(s)
    nA = geom.n_atoms
    assert X.shape == (nA * (nA + 1) // 2, 16)
    bf0 = {0: 0, 1: 15, 2: 20, 3: 25, 4: 40, 5: 45}
    for t in range(X.shape[0]):
        r0, c0, h, onsite = meta[t]
        a = [k for k, v in bf0.items() if v == r0][0]
        b = [k for k, v in bf0.items() if v == c0][0]
        za, zb = geom.Z[a], geom.Z[b]
        assert h == (0 if (za, zb) == (8, 8) else 1 if (za, zb) == (8, 1) else 2)
        d = geom.xyz[b] - geom.xyz[a]
        R = np.linalg.norm(d)
        assert abs(X[t, 0] - R) < 1e-5 * max(1, R)
        if a != b:
            u = d / R
            assert np.allclose(X[t, 1:4], u, atol=1e-6)
            assert np.allclose(X[t, 4:13], np.outer(u, u).ravel(), atol=1e-6)
        else:
            assert onsite == 1 and np.all(X[t, 1:13] == 0)
        assert X[t, 13 + h] == 1.0 and X[t, 13:16].sum() == 1.0


def test_training_and_learned_scf(ctx):
    """A briefly trained network: loss falls, the predicted density is
    symmetric with tr(PS) = N_e, and the SCF started from it reaches the
    core-guess energy within 1e-8 Eh."""
    from paper_1708_00033_gb300 import guess, hf
    data = guess.make_dataset(ctx, 24, lo=2, hi=3)
    model = hf.Model(ctx, guess.init_weights(0))
    losses = guess.train(model, data, steps=400, batch=512, lr=2e-3)
    assert np.mean(losses[-20:]) < 0.3 * np.mean(losses[:5])
    geom = I.water_cluster(3, I.CONFIG_GUESS_EVAL, 99)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10, prim_tau=1e-14)
    P = hf.guess_predict(model, s)
    S, _ = s.one_electron()
    assert np.abs(P - P.T).max() == 0.0
    assert abs(np.trace(P @ S) - int(geom.Z.sum())) < 1e-9
    core = hf.scf(s, e_tol=1e-10, d_tol=1e-7)
    learned = hf.scf(s, e_tol=1e-10, d_tol=1e-7, P_guess=P)
    assert abs(core["energy"] - learned["energy"]) <= 1e-8
