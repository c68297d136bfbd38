"""Full-size parity in the launch configuration bench.py times: the 64-water
cluster (1,600 basis functions), Schwarz 1e-10, the bench's primitive
threshold.  The oracle computes whole J and K shell blocks by definition
(same Schwarz screening, no primitive screening); every element must agree
within 1e-10.  The blocks cover each ordered pair of shell types (s, p, d in
both orders), diagonal shell blocks of each type, blocks of shells on the
same and on distant molecules, and random blocks: over 200 elements."""
import numpy as np
import pytest

from paper_1708_00033_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _blocks(l, atom, rng):
    """Shell pairs (I, J): for every ordered pair of shell types, one block on water 0 and one between
    water 0 and a distant water; a diagonal block of each type; ten random blocks."""
    n = len(l)
    near = {t: [s for s in range(n) if l[s] == t and atom[s] < 3] for t in (0, 1, 2)}  # water 0
    far = {t: [s for s in range(n) if l[s] == t and atom[s] >= 3 * 40] for t in (0, 1, 2)}  # waters 40..63
    out = []
    for ta in (0, 1, 2):
        out.append((near[ta][0], near[ta][0]))
        for tb in (0, 1, 2):
            out.append((near[ta][0], near[tb][-1]))
            out.append((near[ta][-1], far[tb][len(far[tb]) // 2]))
    out += [(int(a), int(b)) for a, b in rng.integers(0, n, size=(10, 2))]
    return out


def test_sixty_four_waters_sampled_blocks(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(64, I.CONFIG_SCF, 0)
    basis = I.synthetic_basis(geom)
    ctx = hf.Context(0)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10, prim_tau=I.BENCH_PRIM_TAU)
    S, _ = s.one_electron()
    G = I.random_orbitals(s.n_bf, 320, I.CONFIG_SCF, 0)
    L = np.linalg.cholesky(G.T @ S @ G)
    P = 2.0 * np.linalg.solve(L, G.T).T @ np.linalg.solve(L, G.T)
    P = 0.5 * (P + P.T)
    out = s.fock_build(torch.from_numpy(P).cuda(), want_J=True, want_K=True)
    J, K = out["J"].cpu().numpy(), out["K"].cpu().numpy()
    mol = oracle_mod.Molecule(geom, basis)
    blocks = _blocks(np.asarray(basis.l), np.asarray(basis.atom), np.random.default_rng(64))
    Jb, Kb = mol.jk_shell_blocks(P, blocks, tau=1e-10)
    n_el = 0
    worst = 0.0
    for (i, j), jb, kb in zip(blocks, Jb, Kb):
        r, c = int(mol.bf0[i]), int(mol.bf0[j])
        dj = np.abs(J[r:r + jb.shape[0], c:c + jb.shape[1]] - jb).max()
        dk = np.abs(K[r:r + kb.shape[0], c:c + kb.shape[1]] - kb).max()
        worst = max(worst, dj, dk)
        assert dj <= 1e-10 and dk <= 1e-10, ((i, j), dj, dk)
        n_el += jb.size
    assert n_el >= 200, n_el
