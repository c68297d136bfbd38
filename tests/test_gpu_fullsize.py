"""Full-size parity in the launch configuration bench.py times: the 64-water
cluster (1,600 basis functions), Schwarz 1e-10, primitive screening 1e-14.
The oracle computes sampled J and K elements one by one (same Schwarz
screening, no primitive screening); they must agree within 1e-10."""
import numpy as np
import pytest

from paper_1708_00033_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_sixty_four_waters_sampled_elements(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(64, I.CONFIG_SCF, 0)
    basis = I.synthetic_basis(geom)
    ctx = hf.Context(0)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10, prim_tau=1e-14)
    S, _ = s.one_electron()
    G = I.random_orbitals(s.n_bf, 320, I.CONFIG_SCF, 0)
    L = np.linalg.cholesky(G.T @ S @ G)
    P = 2.0 * np.linalg.solve(L, G.T).T @ np.linalg.solve(L, G.T)
    P = 0.5 * (P + P.T)
    out = s.fock_build(torch.from_numpy(P).cuda(), want_J=True, want_K=True)
    J, K = out["J"].cpu().numpy(), out["K"].cpu().numpy()
    mol = oracle_mod.Molecule(geom, basis)
    rng = np.random.default_rng(64)
    pairs = [(0, 0), (1599, 1599), (17, 943)] + [tuple(int(x) for x in rng.integers(0, 1600, 2)) for _ in range(5)]
    Jo, Ko = mol.jk_elements(P, pairs, tau=1e-10)
    for t, (a, b) in enumerate(pairs):
        assert abs(J[a, b] - Jo[t]) <= 1e-10, (a, b, J[a, b], Jo[t])
        assert abs(K[a, b] - Ko[t]) <= 1e-10, (a, b, K[a, b], Ko[t])
