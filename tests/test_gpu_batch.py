"""Batched Fock builds (one graph-captured step with persistent class kernels
over many molecules) against per-molecule builds and the oracle."""
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


def _batch_inputs(n_mol, hi=4):
    geoms = [I.batch_cluster(I.CONFIG_BATCH, m, 1, hi) for m in range(n_mol)]
    bases = [I.synthetic_basis(g) for g in geoms]
    return geoms, bases


def _densities(batch, seed=0):
    rng = np.random.default_rng(seed)
    P = np.zeros(int(batch.offsets[-1]))
    for m, n in enumerate(batch.n_bf):
        G = rng.standard_normal((n, max(1, n // 5)))
        P[batch.offsets[m]:batch.offsets[m + 1]] = (0.2 * G @ G.T).ravel()
    return P


@pytest.mark.parametrize("tau", [0.0, 1e-10])
def test_batch_graph_matches_single_builds(ctx, tau, tmp_path):
    import torch
    from paper_1708_00033_gb300 import hf
    geoms, bases = _batch_inputs(7)
    batch = hf.Batch(ctx, geoms, bases, schwarz_tau=tau)
    P = _densities(batch)
    Pd = torch.from_numpy(P).cuda()
    F = torch.empty_like(Pd)
    ms, E = batch.fock_build(Pd, F, energies=True)
    Fs = torch.empty_like(Pd)
    ms_s, E_s = batch.fock_build(Pd, Fs, energies=True, sequential=True)
    assert float((F - Fs).abs().max()) <= 1e-12
    assert np.abs(E - E_s).max() <= 1e-10
    # against independent systems
    for m in range(batch.n_mol):
        s = hf.System(ctx, geoms[m], bases[m], schwarz_tau=tau)
        n = batch.n_bf[m]
        ref = s.fock_build(P[batch.offsets[m]:batch.offsets[m + 1]].reshape(n, n))
        got = F[int(batch.offsets[m]):int(batch.offsets[m + 1])].cpu().numpy().reshape(n, n)
        assert np.abs(got - ref["F"]).max() <= 1e-12
        assert abs(E[m] - ref["E_elec"]) <= 1e-10
    # autotuned graph gives the same result; the cache file round-trips
    cache = str(tmp_path / "tune.txt")
    batch.tune(cache, sample_quartets=20000)
    info = batch.info()
    assert all(b in (64, 128, 256) for b, q in zip(info["block"], info["class_quartets"]) if q > 0)
    F2 = torch.empty_like(Pd)
    batch.fock_build(Pd, F2)
    assert float((F2 - F).abs().max()) <= 1e-12
    batch2 = hf.Batch(ctx, geoms, bases, schwarz_tau=tau)
    batch2.tune(cache)
    assert batch2.info()["block"] == info["block"] and batch2.info()["chunk"] == info["chunk"]


def test_batch_member_vs_oracle(ctx, oracle_mod):
    import torch
    from paper_1708_00033_gb300 import hf
    geoms, bases = _batch_inputs(3, hi=2)
    batch = hf.Batch(ctx, geoms, bases)
    P = _densities(batch, seed=3)
    F = torch.empty(P.shape, dtype=torch.float64, device="cuda")
    batch.fock_build(torch.from_numpy(P).cuda(), F)
    for m in range(3):
        mol = oracle_mod.Molecule(geoms[m], bases[m])
        n = batch.n_bf[m]
        Pm = P[batch.offsets[m]:batch.offsets[m + 1]].reshape(n, n)
        J, K = mol.jk_literal(Pm)
        _, H = mol.core_hamiltonian()
        Fo = oracle_mod.fock_from_jk(H, J, K)
        got = F[int(batch.offsets[m]):int(batch.offsets[m + 1])].cpu().numpy().reshape(n, n)
        assert np.abs(got - Fo).max() <= 1e-10


def test_batch_screened_members_vs_oracle(ctx, oracle_mod):
    """Members of 4 and 8 waters with Schwarz screening at 1e-10 and the bench's primitive threshold, built
    in one graph-captured batched step, against the oracle's screened unique-quartet build (same Schwarz
    rule, no primitive screening) within 1e-10."""
    import torch
    from paper_1708_00033_gb300 import hf
    geoms = [I.water_cluster(4, I.CONFIG_BATCH, 1001), I.water_cluster(8, I.CONFIG_BATCH, 1002),
             I.water_cluster(1, I.CONFIG_BATCH, 1003)]
    bases = [I.synthetic_basis(g) for g in geoms]
    batch = hf.Batch(ctx, geoms, bases, schwarz_tau=1e-10, prim_tau=I.BENCH_PRIM_TAU)
    P = _densities(batch, seed=8)
    F = torch.empty(P.shape, dtype=torch.float64, device="cuda")
    _, E = batch.fock_build(torch.from_numpy(P).cuda(), F, energies=True)
    for m in range(2):
        mol = oracle_mod.Molecule(geoms[m], bases[m])
        n = batch.n_bf[m]
        Pm = P[batch.offsets[m]:batch.offsets[m + 1]].reshape(n, n)
        J, K = mol.jk_unique(Pm, 1e-10)
        _, H = mol.core_hamiltonian()
        Fo = oracle_mod.fock_from_jk(H, J, K)
        got = F[int(batch.offsets[m]):int(batch.offsets[m + 1])].cpu().numpy().reshape(n, n)
        dF = np.abs(got - Fo).max()
        assert dF <= 1e-10
        # E = 1/2 sum P (H + F): an F error of dF moves it by at most 1/2 sum |P| dF, plus the rounding of a
        # sum of n^2 terms of this (large, random-density) energy
        Eo = oracle_mod.electronic_energy(Pm, H, Fo)
        assert abs(E[m] - Eo) <= 0.5 * np.abs(Pm).sum() * dF + 1e-14 * n * abs(Eo)


def test_batch_rejects_bad_density(ctx):
    import torch
    from paper_1708_00033_gb300 import hf
    geoms, bases = _batch_inputs(2, hi=1)
    batch = hf.Batch(ctx, geoms, bases)
    P = _densities(batch)
    P[1] += 0.5  # breaks the symmetry of molecule 0
    with pytest.raises(hf.HFError) as e:
        batch.fock_build(torch.from_numpy(P).cuda(), torch.empty(P.shape, dtype=torch.float64, device="cuda"))
    assert e.value.code == hf.HF_E_INVALID
