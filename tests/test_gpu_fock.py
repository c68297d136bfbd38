"""GPU parity of the Fock build (C-ABI through the binding) against the CPU oracle.

Tolerances: the FP64 path is held to |dF|max <= 1e-10 Eh (the stated target
for plain FP64) when screening is off; with Schwarz screening both sides skip
the same quartets up to round-off in the bounds, so the same 1e-10 holds.
"""
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


def _density(oracle_mod, mol, n_occ, cfg, idx):
    S, _ = mol.core_hamiltonian()
    C = oracle_mod.orthonormalise(I.random_orbitals(mol.n_bf, n_occ, cfg, idx), S)
    return oracle_mod.density_from_orbitals(C)


def _gpu(ctx, geom, basis, P, tau=0.0, cutoff=0.0, device=False):
    import torch
    from paper_1708_00033_gb300 import hf
    s = hf.System(ctx, geom, basis, schwarz_tau=tau, fp32_cutoff=cutoff)
    Pin = torch.from_numpy(P).cuda() if device else P
    out = s.fock_build(Pin, want_J=True, want_K=True, stats=True)
    res = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    res["system"] = s
    return res


def test_one_electron_matrices(ctx, oracle_mod):
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(2, 1, 5)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    S, H = mol.core_hamiltonian()
    s = hf.System(ctx, geom, basis)
    Sg, Hg = s.one_electron()
    assert np.abs(Sg - S).max() < 1e-13
    assert np.abs(Hg - H).max() < 1e-11
    assert abs(s.info["E_nn"] - mol.nuclear_repulsion()) < 1e-11
    Sd, Hd = s.one_electron(device=True)
    assert np.abs(Sd.cpu().numpy() - Sg).max() == 0.0


def test_h2_sto3g(ctx, oracle_mod):
    geom, basis = I.h2_sto3g(1.4)
    mol = oracle_mod.Molecule(geom, basis)
    P = np.array([[0.6, 0.6], [0.6, 0.6]])
    J, K = mol.jk_literal(P)
    r = _gpu(ctx, geom, basis, P)
    assert np.abs(r["J"] - J).max() < 1e-13
    assert np.abs(r["K"] - K).max() < 1e-13


def test_single_water_literal(ctx, oracle_mod):
    geom = I.water_cluster(1, 1, 3)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    P = _density(oracle_mod, mol, 5, 1, 3)
    J, K = mol.jk_literal(P)
    S, H = mol.core_hamiltonian()
    r = _gpu(ctx, geom, basis, P)
    assert np.abs(r["J"] - J).max() < 1e-11
    assert np.abs(r["K"] - K).max() < 1e-11
    F = oracle_mod.fock_from_jk(H, J, K)
    assert np.abs(r["F"] - F).max() < 1e-11
    assert abs(r["E_elec"] - oracle_mod.electronic_energy(P, H, F)) < 1e-10


@pytest.mark.parametrize("device", [False, True])
def test_four_waters_unscreened(ctx, oracle_mod, device):
    """4 waters, 100 basis functions, no screening: every unique quartet."""
    geom = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    P = _density(oracle_mod, mol, 20, I.CONFIG_SINGLE_BUILD, 0)
    J, K = mol.jk_unique(P)
    S, H = mol.core_hamiltonian()
    F = oracle_mod.fock_from_jk(H, J, K)
    r = _gpu(ctx, geom, basis, P, device=device)
    n_sh = basis.n_shells
    n_p = n_sh * (n_sh + 1) // 2
    assert r["stats"]["quartets_fp64"] == n_p * (n_p + 1) // 2 == r["stats"]["quartets_unscreened"]
    assert np.abs(r["F"] - F).max() <= 1e-10
    assert np.abs(r["J"] - J).max() <= 1e-10
    assert np.abs(r["K"] - K).max() <= 1e-10
    assert abs(r["E_elec"] - oracle_mod.electronic_energy(P, H, F)) <= 1e-9


def test_screened_matches_screened_oracle(ctx, oracle_mod):
    geom = I.water_cluster(6, 2, 11)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    P = _density(oracle_mod, mol, 30, 2, 11)
    tau = 1e-10
    J, K = mol.jk_unique(P, tau)
    r = _gpu(ctx, geom, basis, P, tau=tau)
    assert r["stats"]["quartets_fp64"] < r["stats"]["quartets_unscreened"]
    assert abs(r["stats"]["quartets_fp64"] - mol.last_quartets) <= max(2, mol.last_quartets // 100000)
    assert np.abs(r["J"] - J).max() <= 1e-10
    assert np.abs(r["K"] - K).max() <= 1e-10


def test_invalid_density_is_rejected(ctx, oracle_mod):
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(1, 1, 1)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis)
    P = np.eye(s.n_bf)
    P[0, 1] = 0.3  # not symmetric
    with pytest.raises(hf.HFError) as e:
        s.fock_build(P)
    assert e.value.code == hf.HF_E_INVALID
    P = np.eye(s.n_bf)
    P[2, 2] = np.nan
    with pytest.raises(hf.HFError) as e:
        s.fock_build(P)
    assert e.value.code == hf.HF_E_INVALID
    # the system stays usable after a rejected call
    out = s.fock_build(np.eye(s.n_bf))
    assert np.isfinite(out["F"]).all()


def test_invalid_density_device_path_leaves_outputs(ctx):
    """The density check runs on the device and the host reads it once, after the build: a rejected density
    still returns HF_E_INVALID and every device output keeps its previous contents."""
    import torch
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(2, 1, 4)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10)
    N = s.n_bf
    P = torch.eye(N, dtype=torch.float64, device="cuda")
    P[0, 3] = 0.25  # not symmetric
    F, J, K = (torch.full_like(P, 7.0) for _ in range(3))
    with pytest.raises(hf.HFError) as e:
        s.fock_build(P, F=F, J=J, K=K)
    assert e.value.code == hf.HF_E_INVALID
    for t in (F, J, K):
        assert bool((t == 7.0).all())
    P[0, 3] = 0.0
    out = s.fock_build(P, F=F, J=J, K=K, want_J=True, want_K=True)
    ref = s.fock_build(P.cpu().numpy(), want_J=True, want_K=True)
    assert float(np.abs(out["F"].cpu().numpy() - ref["F"]).max()) <= 1e-13


def test_unsupported_basis_is_rejected(ctx):
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(1, 1, 1)
    basis = I.synthetic_basis(geom)
    basis.l = basis.l.copy()
    basis.l[5] = 3
    with pytest.raises(hf.HFError) as e:
        hf.System(ctx, geom, basis)
    assert e.value.code == hf.HF_E_UNSUPPORTED


@pytest.mark.parametrize("prim_tau", [1e-15, 1e-13])
def test_primitive_screening_parity(ctx, oracle_mod, prim_tau):
    """Primitive-pair Schwarz screening changes each integral by at most prim_tau
    per skipped primitive quartet; F must stay within the FP64 tolerance."""
    geom = I.water_cluster(6, 2, 11)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    P = _density(oracle_mod, mol, 30, 2, 11)
    tau = 1e-10
    J, K = mol.jk_unique(P, tau)
    from paper_1708_00033_gb300 import hf
    s = hf.System(ctx, geom, basis, schwarz_tau=tau, prim_tau=prim_tau)
    out = s.fock_build(P, want_J=True, want_K=True, stats=True)
    st = out["stats"]
    assert st["prim_quartets_fp64"] < 81 * st["quartets_fp64"]
    assert np.abs(out["J"] - J).max() <= 1e-10
    assert np.abs(out["K"] - K).max() <= 1e-10


@pytest.mark.parametrize("n_shards", [2, 3])
def test_shards_sum_to_full_build(ctx, oracle_mod, n_shards):
    """hf_fock_build_partial over all shards equals one full build (the
    per-rank partial Fock matrices of the paper's distributed algorithms)."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    P = _density(oracle_mod, mol, 20, I.CONFIG_SINGLE_BUILD, 0)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10, prim_tau=1e-14)
    full = s.fock_build(P, want_J=True, want_K=True)
    parts = [hf.fock_build_partial(s, P, k, n_shards) for k in range(n_shards)]
    # stand-in for an allreduce over ranks: shard 0's partial matrices summed with the others
    sums = {id(parts[0][0]): sum(p[0] for p in parts), id(parts[0][1]): sum(p[1] for p in parts)}
    F, J, K, E = hf.assemble_shards(s, parts[0][0], parts[0][1], lambda a: sums[id(a)], P=P, energy=True)
    assert np.abs(J - full["J"]).max() <= 1e-12
    assert np.abs(K - full["K"]).max() <= 1e-12
    assert np.abs(F - full["F"]).max() <= 1e-12
    assert abs(E - full["E_elec"]) <= 1e-10
    # the same through device tensors (the path an NCCL allreduce uses)
    import torch
    Pd = torch.from_numpy(P).cuda()
    dparts = [hf.fock_build_partial(s, Pd, k, n_shards) for k in range(n_shards)]
    for (Jh, Kh), (Jd, Kd) in zip(parts, dparts):
        assert float(np.abs(Jd.cpu().numpy() - Jh).max()) <= 1e-13
        assert float(np.abs(Kd.cpu().numpy() - Kh).max()) <= 1e-13
    dsum = {id(dparts[0][0]): sum(p[0] for p in dparts), id(dparts[0][1]): sum(p[1] for p in dparts)}
    Fd, _, _, Ed = hf.sharded_fock_build(s, Pd, 0, n_shards, lambda a: dsum[id(a)],
                                         build_partial=lambda *a_: dparts[0])
    assert float((Fd - torch.from_numpy(full["F"]).cuda()).abs().max()) <= 1e-12
    assert abs(Ed - full["E_elec"]) <= 1e-10


def test_fock_assemble_rejects_non_finite(ctx):
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(1, 1, 1)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis)
    N = s.n_bf
    J, K = np.eye(N), np.eye(N)
    F, _ = hf.fock_assemble(s, J, K)
    _, H = s.one_electron()
    assert np.abs(F - (H + 0.5 * np.eye(N))).max() == 0.0
    K[3, 4] = np.inf
    with pytest.raises(hf.HFError) as e:
        hf.fock_assemble(s, J, K)
    assert e.value.code == hf.HF_E_INVALID


@pytest.mark.parametrize("eps,prim_tau", [(1e-3, 0.0), (1e-6, 0.0), (1e-6, 1e-14)])
def test_density_screened_difference_build(ctx, oracle_mod, eps, prim_tau):
    """J and K of a density change dP built with the density-weighted test
    (a quartet is skipped when 4 Q_ab Q_cd max|dP| over the six blocks it
    touches is below the Schwarz threshold; its primitive quartets are
    screened against prim_tau / max|dP|) against the oracle's Schwarz-only
    build of dP.  A skipped quartet changes a J element by less than tau and a
    K element by less than tau/2, a skipped primitive quartet by less than
    4 prim_tau (at most 81 per quartet here), and at most 2 n_pairs quartets
    touch a J element and 4 n_sh^2 a K element: that is the tolerance.
    Per skipped quartet: 4 f X P < tau for J (4 Q_ab Q_cd max|dP| < tau), and
    2 f X P < tau/2 for K; per skipped primitive quartet 4 prim_tau (J) and
    2 prim_tau (K)."""
    from paper_1708_00033_gb300 import hf
    tau = 1e-10
    per_quartet_J = tau + 81 * 4 * prim_tau
    per_quartet_K = 0.5 * tau + 81 * 2 * prim_tau
    geom = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    S, _ = mol.core_hamiltonian()
    C0 = I.random_orbitals(mol.n_bf, 20, I.CONFIG_SINGLE_BUILD, 0)
    C1 = C0 + eps * I.random_orbitals(mol.n_bf, 20, I.CONFIG_SINGLE_BUILD, 1)
    P0 = oracle_mod.density_from_orbitals(oracle_mod.orthonormalise(C0, S))
    P1 = oracle_mod.density_from_orbitals(oracle_mod.orthonormalise(C1, S))
    dP = P1 - P0
    J_ref, K_ref = mol.jk_unique(dP, tau)
    s = hf.System(ctx, geom, basis, schwarz_tau=tau, prim_tau=prim_tau)
    J, K = hf.fock_build_partial(s, dP, density_screen=True, fp64_only=True)
    n_sh = basis.n_shells
    n_pairs = n_sh * (n_sh + 1) // 2
    assert np.abs(J - J_ref).max() <= 2 * n_pairs * per_quartet_J
    assert np.abs(K - K_ref).max() <= 4 * n_sh * n_sh * per_quartet_K
    if prim_tau == 0.0:
        # the same call without the density test is the plain Schwarz-screened build
        J2, K2 = hf.fock_build_partial(s, dP, fp64_only=True)
        assert np.abs(J2 - J_ref).max() <= 1e-12 and np.abs(K2 - K_ref).max() <= 1e-12


@pytest.mark.parametrize("copies", [2, 152, 608])
def test_private_fock_copies(ctx, oracle_mod, copies):
    """Per-block private accumulator copies (the paper's private Fock
    matrices) give the shared-accumulator result up to FP64 summation order,
    and the oracle's within the FP64 tolerance; unscreened 4 waters."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    P = _density(oracle_mod, mol, 20, I.CONFIG_SINGLE_BUILD, 0)
    s = hf.System(ctx, geom, basis)
    shared = s.fock_build(P, want_J=True, want_K=True)
    s.set_fock_copies(copies)
    priv = s.fock_build(P, want_J=True, want_K=True, stats=True)
    for k in ("F", "J", "K"):
        assert np.abs(priv[k] - shared[k]).max() <= 1e-12
    J, K = mol.jk_unique(P)
    assert np.abs(priv["J"] - J).max() <= 1e-10 and np.abs(priv["K"] - K).max() <= 1e-10
    Jp, Kp = hf.fock_build_partial(s, P)
    assert np.abs(Jp - shared["J"]).max() <= 1e-12 and np.abs(Kp - shared["K"]).max() <= 1e-12
    s.set_fock_copies(1)
    again = s.fock_build(P)
    assert np.abs(again["F"] - shared["F"]).max() <= 1e-12
    with pytest.raises(hf.HFError):
        s.set_fock_copies(0)


def test_sp_shell_basis_four_waters_unscreened(ctx, oracle_mod):
    """A split-valence basis with sp (L) shells (s, sp, sp, d on O; s, s on H; 76 functions at 4 waters):
    the library takes the sp shells as given and matches the oracle's unscreened J, K, F and one-electron
    matrices within the FP64 tolerance."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    basis = I.synthetic_sp_basis(geom)
    assert (basis.l == -1).sum() == 8
    mol = oracle_mod.Molecule(geom, basis)
    S, H = mol.core_hamiltonian()
    P = _density(oracle_mod, mol, 20, I.CONFIG_SINGLE_BUILD, 0)
    J, K = mol.jk_literal(P)
    F = oracle_mod.fock_from_jk(H, J, K)
    s = hf.System(ctx, geom, basis)
    assert s.n_bf == mol.n_bf == 76
    Sg, Hg = s.one_electron()
    assert np.abs(Sg - S).max() < 1e-13 and np.abs(Hg - H).max() < 1e-11
    out = s.fock_build(P, want_J=True, want_K=True)
    assert np.abs(out["J"] - J).max() <= 1e-10
    assert np.abs(out["K"] - K).max() <= 1e-10
    assert np.abs(out["F"] - F).max() <= 1e-10
    assert abs(out["E_elec"] - oracle_mod.electronic_energy(P, H, F)) <= 1e-9


def test_sp_shell_basis_scf_vs_oracle(ctx, oracle_mod):
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(2, 2, 8)
    basis = I.synthetic_sp_basis(geom)
    r = hf.scf(hf.System(ctx, geom, basis, schwarz_tau=1e-12), e_tol=1e-11, d_tol=1e-8)
    ref = oracle_mod.scf(oracle_mod.Molecule(geom, basis), e_tol=1e-11, d_tol=1e-8)
    assert r["converged"] and ref.converged
    assert abs(r["energy"] - ref.energy) < 1e-9


def test_rys_quadrature_classes(ctx, oracle_mod):
    """The five classes of total angular momentum L >= 6 have two FP64 kernels: Rys quadrature (4 or 5 nodes
    of the Boys weight) and the Obara-Saika vertical recurrence.  HF_RYS takes Rys for all five,
    HF_OBARA_SAIKA takes Obara-Saika for all, the default takes Rys for (dp|dp), (dd|ds), (dd|dp), (dd|dd).
    All three against the oracle's unscreened J and K (McMurchie-Davidson) at 4 waters within 1e-10 and
    against each other to rounding; then with Schwarz and primitive screening at 8 waters against each
    other."""
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    basis = I.synthetic_basis(geom)
    mol = oracle_mod.Molecule(geom, basis)
    P = _density(oracle_mod, mol, 20, I.CONFIG_SINGLE_BUILD, 0)
    J, K = mol.jk_unique(P)
    s = hf.System(ctx, geom, basis)
    os_ = s.fock_build(P, want_J=True, want_K=True, rys=False)
    ry = s.fock_build(P, want_J=True, want_K=True, rys=True, stats=True)
    de = s.fock_build(P, want_J=True, want_K=True)
    scale = np.abs(os_["F"]).max()
    for r in (os_, ry, de):
        assert np.abs(r["J"] - J).max() <= 1e-10 and np.abs(r["K"] - K).max() <= 1e-10
        assert np.abs(r["F"] - os_["F"]).max() <= 1e-13 * scale
    names = [hf.CLASS_NAMES[c] for c in range(hf.NUM_CLASSES) if ry["stats"]["class_quartets_fp64"][c] > 0]
    assert "(dd|dd)" in names and "(dp|dp)" in names
    g8 = I.water_cluster(8, 2, 3)
    b8 = I.synthetic_basis(g8)
    s8 = hf.System(ctx, g8, b8, schwarz_tau=1e-10, prim_tau=I.BENCH_PRIM_TAU)
    m8 = oracle_mod.Molecule(g8, b8)
    P8 = _density(oracle_mod, m8, 40, 2, 3)
    a = s8.fock_build(P8, want_J=True, want_K=True, rys=False)
    for b in (s8.fock_build(P8, want_J=True, want_K=True, rys=True), s8.fock_build(P8, want_J=True, want_K=True)):
        assert np.abs(a["J"] - b["J"]).max() <= 1e-12 and np.abs(a["K"] - b["K"]).max() <= 1e-12
