"""GPU SCF (orthogonalisation, Jacobi eigensolver, DIIS, density formation)
against the oracle's SCF and against invariants that hold at any size."""
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


@pytest.mark.parametrize("n", [1, 2, 5, 64, 257, 600])
def test_eigh_vs_library_routine(ctx, n):
    from paper_1708_00033_gb300 import hf
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n))
    A = G + G.T
    A[0, 0] += 3.0
    w, V = hf.eigh(ctx, A)
    w_ref = np.linalg.eigvalsh(A)
    scale = np.abs(w_ref).max()
    assert np.abs(w - w_ref).max() <= 1e-12 * scale
    assert np.abs(A @ V - V * w).max() <= 1e-11 * scale
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12


def test_eigh_degenerate_and_diagonal(ctx):
    from paper_1708_00033_gb300 import hf
    A = np.diag([3.0, 1.0, 1.0, -2.0, 5.0, 1.0])
    w, V = hf.eigh(ctx, A)
    assert np.allclose(w, [-2.0, 1.0, 1.0, 1.0, 3.0, 5.0], atol=1e-15)
    assert np.abs(A @ V - V * w).max() < 1e-14


def test_scf_h2_textbook(ctx, oracle_mod):
    from paper_1708_00033_gb300 import hf
    geom, basis = I.h2_sto3g(1.4)
    s = hf.System(ctx, geom, basis)
    r = hf.scf(s, e_tol=1e-12, d_tol=1e-10)
    assert r["converged"]
    ref = oracle_mod.scf(oracle_mod.Molecule(geom, basis), e_tol=1e-12, d_tol=1e-10)
    assert abs(r["energy"] - ref.energy) < 1e-10
    assert abs(r["energy"] - (-1.1167)) <= 0.5e-4


_ORACLE_SCF = {}


def _oracle_scf(oracle_mod, nw, seed):
    """The oracle's unscreened SCF of a cluster, converged tightly (cached per cluster)."""
    if (nw, seed) not in _ORACLE_SCF:
        geom = I.water_cluster(nw, 2, seed)
        basis = I.synthetic_basis(geom)
        ref = oracle_mod.scf(oracle_mod.Molecule(geom, basis), e_tol=1e-11, d_tol=1e-8)
        assert ref.converged
        _ORACLE_SCF[(nw, seed)] = ref
    return _ORACLE_SCF[(nw, seed)]


@pytest.mark.parametrize("nw,seed", [(1, 2), (2, 4)])
def test_scf_vs_oracle(ctx, oracle_mod, nw, seed):
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(nw, 2, seed)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis)
    r = hf.scf(s, e_tol=1e-11, d_tol=1e-8)
    ref = _oracle_scf(oracle_mod, nw, seed)
    assert r["converged"]
    assert abs(r["energy"] - ref.energy) < 1e-9
    assert np.abs(r["P"] - ref.P).max() < 1e-6
    assert np.abs(r["eps"][: len(ref.eps)] - ref.eps).max() < 1e-6


@pytest.mark.parametrize("nw,seed", [(2, 4), (3, 6)])
def test_mixed_scf_vs_oracle(ctx, oracle_mod, nw, seed):
    """Mixed-then-FP64 SCF (FP32 integrals for Q_ij Q_kl < 1e-4 until |dE| < 1e-5, FP64 builds from
    then on, convergence declared on FP64 builds only) from the core-Hamiltonian guess: its energy is the
    plain method's, within 1e-8 Eh of the oracle's SCF and 1e-9 of the plain GPU SCF."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(nw, 2, seed)
    basis = I.synthetic_basis(geom)
    plain = hf.scf(hf.System(ctx, geom, basis), e_tol=1e-11, d_tol=1e-8)
    sm = hf.System(ctx, geom, basis, fp32_cutoff=1e-4)
    assert sm.info["quartets_fp32"] > 0
    mixed = hf.scf(sm, e_tol=1e-11, d_tol=1e-8)
    assert plain["converged"] and mixed["converged"]
    assert 0 < mixed["mixed_iterations"] < mixed["iterations"]  # the last builds were FP64 only
    ref = _oracle_scf(oracle_mod, nw, seed)
    assert abs(mixed["energy"] - ref.energy) <= 1e-8
    assert abs(mixed["energy"] - plain["energy"]) <= 1e-9
    assert np.abs(mixed["P"] - plain["P"]).max() < 1e-6


def test_mixed_scf_from_a_given_density(ctx):
    """The mixed phase also runs from a supplied starting density (the learned guess's path): started from
    a slightly perturbed converged density it still switches to FP64 and lands on the plain energy."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(3, 2, 6)
    basis = I.synthetic_basis(geom)
    plain = hf.scf(hf.System(ctx, geom, basis), e_tol=1e-11, d_tol=1e-8)
    rng = np.random.default_rng(2)
    D = rng.standard_normal(plain["P"].shape) * 1e-2
    Pg = plain["P"] + 0.5 * (D + D.T)
    mixed = hf.scf(hf.System(ctx, geom, basis, fp32_cutoff=1e-4), e_tol=1e-11, d_tol=1e-8, P_guess=Pg)
    assert mixed["converged"] and 0 < mixed["mixed_iterations"] < mixed["iterations"]
    assert abs(mixed["energy"] - plain["energy"]) <= 1e-9


def test_scf_invariants_sixteen_waters(ctx):
    """400 basis functions, Schwarz 1e-10: properties any converged closed-shell SCF has."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(16, 2, 0)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10)
    r = hf.scf(s)
    assert r["converged"]
    S, H = s.one_electron()
    P = r["P"]
    n_el = int(geom.Z.sum())
    assert abs(np.trace(P @ S) - n_el) < 1e-8
    assert np.abs(P @ S @ P - 2.0 * P).max() < 1e-6  # idempotency of the total density
    F = s.fock_build(P)["F"]
    comm = F @ P @ S - S @ P @ F
    assert np.abs(comm).max() < 1e-4
    assert r["energy"] <= r["energies"][0] + 1e-10  # below the core-guess iteration
    assert np.all(np.diff(r["eps"]) >= -1e-12)


def test_scf_reports_nonconvergence(ctx):
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(2, 2, 4)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis)
    r = hf.scf(s, max_iter=2, raise_on_noconv=False)
    assert r["status"] == hf.HF_E_NOCONV and not r["converged"] and r["iterations"] == 2


@pytest.mark.parametrize("rebuild_every", [3, 8])
def test_incremental_scf_matches_plain(ctx, rebuild_every):
    """Incremental SCF (J, K accumulated from density-screened builds of
    P_k - P_ref, full rebuild every few iterations and before convergence is
    declared) converges to the plain SCF's energy and density."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(8, 2, 3)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10)
    # converged tightly, so that both densities are within ~1e-7 of the exact solution
    plain = hf.scf(s, e_tol=1e-11, d_tol=1e-8)
    inc = hf.scf(s, e_tol=1e-11, d_tol=1e-8, incremental=True, rebuild_every=rebuild_every)
    assert plain["converged"] and inc["converged"]
    assert plain["full_builds"] == plain["iterations"]
    assert 1 <= inc["full_builds"] < inc["iterations"]
    assert abs(inc["energy"] - plain["energy"]) < 1e-9
    assert np.abs(inc["P"] - plain["P"]).max() < 1e-6
