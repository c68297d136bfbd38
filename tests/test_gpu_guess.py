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
    w0 = I.guess_init_weights(3)
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


def test_targets_match_density_blocks(ctx):
    """hf_guess_targets places each atom pair's density block in its head's outputs, mask 1 there and 0
    elsewhere (checked against slicing the density by the features' metadata)."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(3, 5, 2)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis)
    N = s.n_bf
    rng = np.random.default_rng(1)
    P = rng.standard_normal((N, N))
    P = P + P.T
    T, M = hf.guess_targets(s, P)
    _, meta = hf.guess_features(s)
    off, shape = (0, 225, 300), ((15, 15), (15, 5), (5, 5))
    assert T.shape == M.shape == (meta.shape[0], 325)
    for t in range(meta.shape[0]):
        r0, c0, h, _ = (int(x) for x in meta[t])
        nr, nc = shape[h]
        want = np.zeros(325, dtype=np.float32)
        want[off[h]:off[h] + nr * nc] = P[r0:r0 + nr, c0:c0 + nc].ravel()
        assert np.array_equal(T[t], want)
        assert M[t].sum() == nr * nc and np.all(M[t, off[h]:off[h] + nr * nc] == 1.0)


def test_library_training_loop(ctx):
    """hf_guess_train: the loss falls; the same seed gives the same weights; the first step equals one
    hf_model_train_step on the minibatch the SplitMix64 draw selects."""
    import torch
    from paper_1708_00033_gb300 import hf
    rng = np.random.default_rng(4)
    n = 700
    X = rng.standard_normal((n, 16)).astype(np.float32)
    W = rng.standard_normal((16, 325)).astype(np.float32) * 0.3
    T = np.tanh(X @ W).astype(np.float32)
    M = (rng.random((n, 325)) < 0.5).astype(np.float32)
    dev = torch.device("cuda")
    Xd, Td, Md = (torch.from_numpy(a).to(dev) for a in (X, T, M))
    w0 = I.guess_init_weights(1)
    a, b = hf.Model(ctx, w0), hf.Model(ctx, w0)
    la = hf.guess_train(a, Xd, Td, Md, steps=300, batch=128, lr=2e-3, seed=9)
    lb = hf.guess_train(b, Xd, Td, Md, steps=300, batch=128, lr=2e-3, seed=9)
    assert np.array_equal(la, lb) and np.array_equal(a.weights(), b.weights())
    assert la[-20:].mean() < 0.5 * la[:5].mean()

    def splitmix64(seed, i):
        m = (1 << 64) - 1
        z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & m
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        return z ^ (z >> 31)

    rows = [splitmix64(9, j) % n for j in range(128)]
    c, d = hf.Model(ctx, w0), hf.Model(ctx, w0)
    l1 = hf.guess_train(c, Xd, Td, Md, steps=1, batch=128, lr=2e-3, seed=9)
    xb, tb, mb = (torch.from_numpy(np.ascontiguousarray(a_[rows])).to(dev) for a_ in (X, T, M))
    l2 = d.train_step(xb, tb, mb, 2e-3)
    assert abs(float(l1[0]) - l2) <= 1e-6 * max(1.0, l2)
    assert np.abs(c.weights() - d.weights()).max() <= 1e-7


def test_training_and_learned_scf(ctx):
    """A briefly trained network: loss falls, the predicted density is
    symmetric with tr(PS) = N_e, and the SCF started from it reaches the
    core-guess energy within 1e-8 Eh."""
    from paper_1708_00033_gb300 import guess, hf
    data = guess.make_dataset(ctx, 24, lo=2, hi=3)
    model = hf.Model(ctx, I.guess_init_weights(0))
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
    # mixed precision from the learned guess: FP32 phase, then FP64 builds to the same energy
    sm = hf.System(ctx, geom, basis, schwarz_tau=1e-10, prim_tau=1e-14, fp32_cutoff=1e-4)
    mixed = hf.scf(sm, e_tol=1e-10, d_tol=1e-7, P_guess=P)
    assert mixed["converged"] and 0 < mixed["mixed_iterations"] < mixed["iterations"]
    assert abs(mixed["energy"] - core["energy"]) <= 1e-8


def test_trained_network_gain():
    """The shipped network (trained by train_guess.py on plain-SCF densities of 2-8 water clusters) against
    the method without it, on held-out clusters of 10-16 waters (seeds (6, m), never trained on, larger
    than any training cluster): the SCF from the learned density needs fewer iterations than the SCF from
    the core-Hamiltonian guess on every cluster, at most 0.7 times as many on average, and converges to the
    same energy within 1e-8 Eh."""
    import os
    from paper_1708_00033_gb300 import guess, hf
    assert os.path.exists(guess.WEIGHTS_PATH), "trained weights are missing"
    w, meta = guess.load_weights()
    ctx = hf.Context(0)
    model = hf.Model(ctx, w)
    core_it, learned_it = [], []
    for m, nw in enumerate((10, 12, 14, 16)):
        geom = I.water_cluster(nw, I.CONFIG_GUESS_EVAL, 100 + m)
        basis = I.synthetic_basis(geom)
        s = hf.System(ctx, geom, basis, schwarz_tau=1e-10, prim_tau=I.BENCH_PRIM_TAU)
        core = hf.scf(s, e_tol=1e-9, d_tol=1e-6)
        Pg = guess.predict_or_none(model, s)
        assert Pg is not None
        learned = hf.scf(s, e_tol=1e-9, d_tol=1e-6, P_guess=Pg)
        assert core["converged"] and learned["converged"]
        assert abs(core["energy"] - learned["energy"]) <= 1e-8
        assert learned["iterations"] < core["iterations"], (nw, learned["iterations"], core["iterations"])
        core_it.append(core["iterations"])
        learned_it.append(learned["iterations"])
    assert np.mean(learned_it) <= 0.7 * np.mean(core_it), (core_it, learned_it)
