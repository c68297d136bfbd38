"""Pins of the CPU oracle against values fixed outside it.

Each check is chosen so that a plausible slip in the oracle (a dropped
recurrence term, a wrong sign or index, a transposed operand, a missing
normalisation or degeneracy factor) fails at least one of them:
  * Boys function vs scipy's regularised incomplete gamma function;
  * primitive (ss|ss) vs the electrostatic energy of two Gaussian charge
    clouds, Q1 Q2 erf(sqrt(rho) R)/R (Gaussian product theorem + Gauss's law);
  * p and d primitives vs derivative identities of that closed form
    (x_A g = (1/2a) d/dA_x g; x_A^2 g = (d^2/dA_x^2 + 2a) g / 4a^2),
    evaluated with mpmath at 30 digits;
  * the same identities for S, T and V on closed s-s forms;
  * H2/STO-3G at 1.4 bohr vs the textbook's printed integrals and energy;
  * 8-fold permutational symmetry and the Schwarz inequality;
  * literal ordered-index J/K vs the unique-quartet digestion of Eq. 1a-1f;
  * tr(PS) = N_e, diag S = 1, energy invariance under rigid motions and atom
    relabelling, and the variational bound.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_1708_00033_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Boys --
def test_boys_zero_argument(oracle_mod):
    F = oracle_mod.boys(12, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(13)], rtol=0, atol=1e-16)


@pytest.mark.parametrize("T", [1e-9, 1e-3, 0.3, 1.0, 4.7, 12.0, 29.9, 39.999, 40.0, 41.5, 75.0, 300.0])
def test_boys_vs_incomplete_gamma(oracle_mod, T):
    """F_m(T) = gamma_lower(m + 1/2, T) / (2 T^(m + 1/2)), evaluated by mpmath at 30 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    F = oracle_mod.boys(12, T)
    for m in range(13):
        a = mp.mpf(m) + mp.mpf(1) / 2
        ref = float(mp.gammainc(a, 0, mp.mpf(T)) / (2 * mp.mpf(T) ** a))
        assert abs(F[m] - ref) <= 4e-15 * abs(ref), (m, T, F[m], ref)


# ------------------------------------------------- closed-form integrals --
def _cloud_ssss(mp, A, B, C, D, a, b, c, d):
    """[ss|ss] as the Coulomb energy of two spherical Gaussian charge clouds."""
    p, q = a + b, c + d
    P = [(a * A[i] + b * B[i]) / p for i in range(3)]
    Q = [(c * C[i] + d * D[i]) / q for i in range(3)]
    Kab = mp.exp(-a * b / p * sum((A[i] - B[i]) ** 2 for i in range(3)))
    Kcd = mp.exp(-c * d / q * sum((C[i] - D[i]) ** 2 for i in range(3)))
    q1 = Kab * (mp.pi / p) ** 1.5
    q2 = Kcd * (mp.pi / q) ** 1.5
    R = mp.sqrt(sum((P[i] - Q[i]) ** 2 for i in range(3)))
    rho = p * q / (p + q)
    if R == 0:
        return q1 * q2 * 2 * mp.sqrt(rho / mp.pi)
    return q1 * q2 * mp.erf(mp.sqrt(rho) * R) / R


def test_ssss_closed_form(oracle_mod):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    rng = np.random.default_rng(11)
    for _ in range(40):
        cen = rng.uniform(-2, 2, size=(4, 3))
        ex = rng.uniform(0.1, 50.0, size=4)
        ref = float(_cloud_ssss(mp.mp, *[[mp.mpf(float(v)) for v in c] for c in cen], *[mp.mpf(float(e)) for e in ex]))
        got = oracle_mod.eri_primitive([0, 0, 0], ex[0], cen[0], [0, 0, 0], ex[1], cen[1],
                                       [0, 0, 0], ex[2], cen[2], [0, 0, 0], ex[3], cen[3])
        assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-300
    # coincident charge centres (R = 0 limit)
    c0 = [0.2, -0.1, 0.4]
    ref = float(_cloud_ssss(mp.mp, *[[mp.mpf(v) for v in c0]] * 4, mp.mpf(1), mp.mpf(2), mp.mpf(3), mp.mpf(4)))
    got = oracle_mod.eri_primitive([0, 0, 0], 1.0, c0, [0, 0, 0], 2.0, c0, [0, 0, 0], 3.0, c0, [0, 0, 0], 4.0, c0)
    assert abs(got - ref) <= 1e-13 * ref


def _power_terms(power, a):
    """Operator turning an s primitive on a centre into x^n: list of (order, coef)."""
    if power == 0:
        return [(0, 1.0)]
    if power == 1:
        return [(1, 1.0 / (2 * a))]
    if power == 2:
        return [(2, 1.0 / (4 * a * a)), (0, 2 * a / (4 * a * a))]
    raise ValueError


def _apply_derivatives(mp, f, point, powers, exps):
    """sum over operator expansions of mpmath partial derivatives of f(point)."""
    per_coord = []
    for centre in range(len(exps)):
        for axis in range(3):
            per_coord.append(_power_terms(powers[centre][axis], exps[centre]))
    total = mp.mpf(0)
    for combo in itertools.product(*per_coord):
        orders = tuple(o for o, _ in combo)
        coef = mp.mpf(1)
        for _, cf in combo:
            coef *= cf
        total += coef * (mp.diff(f, tuple(point), orders) if any(orders) else f(*point))
    return total


CARTS = {0: [(0, 0, 0)], 1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
         2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]}

ERI_CASES = [
    ((1, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0)),
    ((0, 0, 0), (0, 1, 0), (0, 0, 0), (0, 0, 0)),
    ((0, 0, 0), (0, 0, 0), (0, 0, 1), (0, 0, 0)),
    ((0, 0, 0), (0, 0, 0), (0, 0, 0), (1, 0, 0)),
    ((2, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0)),
    ((1, 1, 0), (0, 0, 0), (0, 0, 0), (0, 0, 0)),
    ((0, 0, 0), (0, 0, 0), (0, 0, 0), (0, 0, 2)),
    ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 0, 0)),
    ((2, 0, 0), (1, 1, 0), (0, 0, 0), (0, 0, 1)),
    ((0, 2, 0), (0, 0, 1), (1, 0, 1), (0, 0, 0)),
    ((0, 1, 1), (1, 0, 0), (0, 0, 2), (0, 1, 0)),
]


@pytest.mark.parametrize("pw", ERI_CASES)
def test_eri_derivative_identities(oracle_mod, pw):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    cen = [[0.1, -0.2, 0.3], [0.9, 0.4, -0.5], [-0.6, 1.1, 0.2], [0.3, -0.8, 1.2]]
    ex = [0.9, 1.3, 0.7, 1.6]
    mex = [mp.mpf(e) for e in ex]

    def f(*x):
        return _cloud_ssss(mp.mp, x[0:3], x[3:6], x[6:9], x[9:12], *mex)

    point = [mp.mpf(v) for c in cen for v in c]
    ref = float(_apply_derivatives(mp.mp, f, point, pw, mex))
    got = oracle_mod.eri_primitive(pw[0], ex[0], cen[0], pw[1], ex[1], cen[1], pw[2], ex[2], cen[2], pw[3], ex[3], cen[3])
    assert abs(got - ref) <= 1e-10 * max(abs(ref), 1e-6), (pw, got, ref)


ONEE_CASES = [((0, 0, 0), (0, 0, 0)), ((1, 0, 0), (0, 0, 0)), ((0, 0, 0), (0, 1, 0)), ((2, 0, 0), (0, 0, 0)),
              ((1, 1, 0), (0, 0, 1)), ((0, 0, 2), (2, 0, 0)), ((0, 1, 1), (1, 0, 1))]


@pytest.mark.parametrize("pw", ONEE_CASES)
def test_one_electron_derivative_identities(oracle_mod, pw):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    A, B, C = [0.2, -0.3, 0.1], [-0.5, 0.7, 0.9], [0.4, 0.5, -0.6]
    a, b, Zc = 0.8, 1.7, 3.0
    ma, mb = mp.mpf(a), mp.mpf(b)

    def s_ss(*x):
        Ax, Bx = x[0:3], x[3:6]
        p = ma + mb
        mu = ma * mb / p
        return (mp.pi / p) ** 1.5 * mp.exp(-mu * sum((Ax[i] - Bx[i]) ** 2 for i in range(3)))

    def t_ss(*x):
        Ax, Bx = x[0:3], x[3:6]
        p = ma + mb
        mu = ma * mb / p
        R2 = sum((Ax[i] - Bx[i]) ** 2 for i in range(3))
        return mu * (3 - 2 * mu * R2) * (mp.pi / p) ** 1.5 * mp.exp(-mu * R2)

    def v_ss(*x):
        Ax, Bx = x[0:3], x[3:6]
        p = ma + mb
        mu = ma * mb / p
        R2 = sum((Ax[i] - Bx[i]) ** 2 for i in range(3))
        P = [(ma * Ax[i] + mb * Bx[i]) / p for i in range(3)]
        t = p * sum((P[i] - C[i]) ** 2 for i in range(3))
        F0 = mp.sqrt(mp.pi / t) * mp.erf(mp.sqrt(t)) / 2
        return -Zc * 2 * mp.pi / p * mp.exp(-mu * R2) * F0

    point = [mp.mpf(v) for v in A + B]
    got = oracle_mod.one_electron_primitive(pw[0], a, A, pw[1], b, B, Zc, C)
    for k, fn in enumerate((s_ss, t_ss, v_ss)):
        ref = float(_apply_derivatives(mp.mp, fn, point, pw, [ma, mb]))
        assert abs(got[k] - ref) <= 1e-10 * max(abs(ref), 1e-6), (pw, k, got[k], ref)


# ------------------------------------------------------------- textbook --
def test_h2_sto3g_textbook(oracle_mod):
    ref = json.load(open(os.path.join(GOLDEN, "h2_sto3g_szabo_ostlund.json")))
    g, b = I.h2_sto3g(ref["r_bohr"])
    m = oracle_mod.Molecule(g, b)
    S, H = m.core_hamiltonian()
    eri = m.eri_full()
    half = 0.5 * 10.0 ** (-ref["printed_decimals"]) + 1e-12
    assert abs(S[0, 1] - ref["S12"]) <= half
    assert abs(eri[0, 0, 0, 0] - ref["eri_11_11"]) <= half
    assert abs(eri[0, 0, 1, 1] - ref["eri_11_22"]) <= half
    assert abs(eri[1, 0, 0, 0] - ref["eri_21_11"]) <= half
    assert abs(eri[1, 0, 1, 0] - ref["eri_21_21"]) <= half
    r = oracle_mod.scf(m, e_tol=1e-12, d_tol=1e-10)
    assert r.converged
    assert abs(r.energy - ref["E_total"]) <= half
    assert abs(r.energy - m.nuclear_repulsion() - ref["E_elec"]) <= half


# ----------------------------------------------------- symmetry, bounds --
@pytest.fixture(scope="module")
def dimer(oracle_mod):
    g = I.water_cluster(2, 1, 7)
    b = I.synthetic_basis(g)
    return oracle_mod.Molecule(g, b)


def test_diag_overlap_is_one(dimer):
    S, _ = dimer.core_hamiltonian()
    assert np.allclose(np.diag(S), 1.0, atol=1e-14)
    assert np.allclose(S, S.T, atol=1e-15)


def test_eight_fold_symmetry_and_schwarz(dimer):
    rng = np.random.default_rng(3)
    Q = dimer.schwarz()
    n = dimer.n_shells
    for _ in range(25):
        i, j, k, l = (int(x) for x in rng.integers(0, n, size=4))
        x = dimer.eri_shell_quartet(i, j, k, l)
        assert np.allclose(x, dimer.eri_shell_quartet(j, i, k, l).transpose(1, 0, 2, 3), atol=1e-13)
        assert np.allclose(x, dimer.eri_shell_quartet(i, j, l, k).transpose(0, 1, 3, 2), atol=1e-13)
        assert np.allclose(x, dimer.eri_shell_quartet(k, l, i, j).transpose(2, 3, 0, 1), atol=1e-13)
        assert np.all(np.abs(x) <= Q[i, j] * Q[k, l] * (1 + 1e-12) + 1e-15)


def test_trace_PS_equals_electron_count(dimer, oracle_mod):
    S, _ = dimer.core_hamiltonian()
    G = I.random_orbitals(dimer.n_bf, dimer.n_electrons // 2, 1, 0)
    C = oracle_mod.orthonormalise(G, S)
    P = oracle_mod.density_from_orbitals(C)
    assert abs(np.trace(P @ S) - dimer.n_electrons) < 1e-10


def test_jk_literal_vs_numpy_and_unique(oracle_mod):
    g = I.water_cluster(1, 1, 3)
    b = I.synthetic_basis(g)
    m = oracle_mod.Molecule(g, b)
    S, _ = m.core_hamiltonian()
    C = oracle_mod.orthonormalise(I.random_orbitals(m.n_bf, 5, 1, 3), S)
    P = oracle_mod.density_from_orbitals(C)
    eri = m.eri_full()
    Jn = np.einsum("ijkl,kl->ij", eri, P)
    Kn = np.einsum("ikjl,kl->ij", eri, P)
    Jl, Kl = m.jk_literal(P)
    Ju, Ku = m.jk_unique(P)
    assert np.abs(Jl - Jn).max() < 1e-12 and np.abs(Kl - Kn).max() < 1e-12
    assert np.abs(Ju - Jl).max() < 1e-12 and np.abs(Ku - Kl).max() < 1e-12
    # a non-symmetric-looking density must still give the symmetric J/K of its symmetric part
    el = m.jk_elements(P, [(0, 0), (3, 17), (24, 1)])
    for t, (mu, nu) in enumerate([(0, 0), (3, 17), (24, 1)]):
        assert abs(el[0][t] - Jl[mu, nu]) < 1e-12 and abs(el[1][t] - Kl[mu, nu]) < 1e-12


def test_unique_quartet_count(oracle_mod, dimer):
    """Algorithm 1 with the canonical l bound visits n_p(n_p+1)/2 quartets."""
    P = np.eye(dimer.n_bf)
    dimer.jk_unique(P)
    n = dimer.n_shells
    n_p = n * (n + 1) // 2
    assert dimer.last_quartets == n_p * (n_p + 1) // 2


def test_screening_error_is_small(oracle_mod, dimer):
    S, _ = dimer.core_hamiltonian()
    C = oracle_mod.orthonormalise(I.random_orbitals(dimer.n_bf, 10, 1, 4), S)
    P = oracle_mod.density_from_orbitals(C)
    J0, K0 = dimer.jk_unique(P, 0.0)
    J1, K1 = dimer.jk_unique(P, 1e-10)
    assert np.abs(J1 - J0).max() < 1e-8 and np.abs(K1 - K0).max() < 1e-8


# ---------------------------------------------------------------- SCF --
def _rotation(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_energy_invariance_and_variational_bound(oracle_mod):
    g = I.water_cluster(2, 1, 9)
    b = I.synthetic_basis(g)
    e_ref = oracle_mod.scf(oracle_mod.Molecule(g, b), e_tol=1e-11, d_tol=1e-8)
    assert e_ref.converged
    # variational: converged energy below the first (core-guess) iteration
    assert e_ref.energy <= e_ref.history[0][0] + 1e-12
    R = _rotation([0.3, -1.0, 0.5], 0.77)
    moved = I.Geometry(Z=g.Z.copy(), xyz=g.xyz @ R.T + np.array([1.5, -2.0, 0.25]))
    e_rot = oracle_mod.scf(oracle_mod.Molecule(moved, b), e_tol=1e-11, d_tol=1e-8)
    assert abs(e_rot.energy - e_ref.energy) < 1e-9
    perm = np.array([3, 4, 5, 0, 1, 2])  # swap the two waters
    inv = np.argsort(perm)
    pg = I.Geometry(Z=g.Z[perm].copy(), xyz=g.xyz[perm].copy())
    pb = I.synthetic_basis(pg)
    e_perm = oracle_mod.scf(oracle_mod.Molecule(pg, pb), e_tol=1e-11, d_tol=1e-8)
    assert abs(e_perm.energy - e_ref.energy) < 1e-9
    assert inv is not None


@pytest.mark.slow
def test_literal_vs_unique_four_waters(oracle_mod):
    """Unique-quartet digestion (used for >100 BF) agrees with the literal sums at 100 BF."""
    g = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    b = I.synthetic_basis(g)
    m = oracle_mod.Molecule(g, b)
    S, _ = m.core_hamiltonian()
    P = oracle_mod.density_from_orbitals(oracle_mod.orthonormalise(I.random_orbitals(m.n_bf, 20, 1, 0), S))
    Ju, Ku = m.jk_unique(P)
    Jl, Kl = m.jk_literal(P)
    assert np.abs(Ju - Jl).max() < 1e-11 and np.abs(Ku - Kl).max() < 1e-11


@pytest.mark.parametrize("tau", [0.0, 1e-10])
def test_strided_sample_partitions_the_unique_loop(oracle_mod, dimer, tau):
    """The CPU-baseline sample (every stride-th bra pair) partitions Algorithm 1's
    unique-quartet loop: over all offsets the evaluated quartets add up to the full
    loop's count and the spanned quartets to n_p (n_p + 1) / 2."""
    n_sh = dimer.n_shells
    n_p = n_sh * (n_sh + 1) // 2
    S, _ = dimer.core_hamiltonian()
    P = oracle_mod.density_from_orbitals(oracle_mod.orthonormalise(I.random_orbitals(dimer.n_bf, 10, 1, 0), S))
    dimer.jk_unique(P, tau)
    full = dimer.last_quartets
    stride = 7
    got = [dimer.jk_unique_sample(P, tau, stride, off) for off in range(stride)]
    assert sum(n for n, _ in got) == full
    assert sum(u for _, u in got) == n_p * (n_p + 1) // 2
    if tau == 0.0:
        assert full == n_p * (n_p + 1) // 2


def test_shell_blocks_vs_literal(oracle_mod):
    """Whole J/K shell blocks by definition equal the literal ordered-index sums (themselves pinned to
    numpy einsum above), on every shell pair of one water."""
    g = I.water_cluster(1, 1, 3)
    b = I.synthetic_basis(g)
    m = oracle_mod.Molecule(g, b)
    S, _ = m.core_hamiltonian()
    P = oracle_mod.density_from_orbitals(oracle_mod.orthonormalise(I.random_orbitals(m.n_bf, 5, 1, 3), S))
    Jl, Kl = m.jk_literal(P)
    blocks = [(i, j) for i in range(m.n_shells) for j in range(m.n_shells)]
    Jb, Kb = m.jk_shell_blocks(P, blocks)
    for (i, j), jb, kb in zip(blocks, Jb, Kb):
        r, c = int(m.bf0[i]), int(m.bf0[j])
        assert np.abs(jb - Jl[r:r + jb.shape[0], c:c + jb.shape[1]]).max() < 1e-12
        assert np.abs(kb - Kl[r:r + kb.shape[0], c:c + kb.shape[1]]).max() < 1e-12


def test_screened_elements_and_blocks_vs_unique(oracle_mod):
    """With Schwarz screening, the by-definition elements and shell blocks leave out exactly the integrals
    the unique-quartet build leaves out: the Coulomb integral (mu nu|lam sig) by Q_IJ Q_kl and the exchange
    integral (mu lam|nu sig) by Q_Ik Q_Jl.  A threshold large enough to change J and K makes a wrong pair
    index visible."""
    g = I.water_cluster(3, 2, 5)
    b = I.synthetic_basis(g)
    m = oracle_mod.Molecule(g, b)
    S, _ = m.core_hamiltonian()
    P = oracle_mod.density_from_orbitals(oracle_mod.orthonormalise(I.random_orbitals(m.n_bf, 15, 2, 5), S))
    tau = 1e-6
    J0, K0 = m.jk_unique(P)
    Ju, Ku = m.jk_unique(P, tau)
    assert np.abs(Ju - J0).max() > 1e-8 and np.abs(Ku - K0).max() > 1e-8  # the threshold matters here
    rng = np.random.default_rng(11)
    blocks = [(int(x), int(y)) for x, y in rng.integers(0, m.n_shells, size=(16, 2))] + [(0, 0), (5, 5)]
    Jb, Kb = m.jk_shell_blocks(P, blocks, tau=tau)
    for (i, j), jb, kb in zip(blocks, Jb, Kb):
        r, c = int(m.bf0[i]), int(m.bf0[j])
        assert np.abs(jb - Ju[r:r + jb.shape[0], c:c + jb.shape[1]]).max() < 1e-12
        assert np.abs(kb - Ku[r:r + kb.shape[0], c:c + kb.shape[1]]).max() < 1e-12
    pairs = [(int(x), int(y)) for x, y in rng.integers(0, m.n_bf, size=(12, 2))]
    Je, Ke = m.jk_elements(P, pairs, tau=tau)
    for t, (mu, nu) in enumerate(pairs):
        assert abs(Je[t] - Ju[mu, nu]) < 1e-12 and abs(Ke[t] - Ku[mu, nu]) < 1e-12


def test_sp_shell_is_an_s_and_a_p_shell(oracle_mod):
    """An sp shell is by definition an s and a p shell with the same exponents and their own coefficients:
    a basis written with sp shells gives the same S, H and SCF energy as the same shells written out
    separately by hand (s coefficients in the s shell, p coefficients in the p shell)."""
    g = I.water_cluster(1, 2, 1)
    sp = I.synthetic_sp_basis(g)
    atom, l, nprim, exps, coefs = [], [], [], [], []
    o = 0
    for s_ in range(sp.n_shells):
        n = int(sp.nprim[s_])
        parts = [(0, sp.coefs), (1, sp.coefs_p)] if sp.l[s_] == -1 else [(int(sp.l[s_]), sp.coefs)]
        for lq, c in parts:
            atom.append(int(sp.atom[s_]))
            l.append(lq)
            nprim.append(n)
            exps += list(sp.exps[o:o + n])
            coefs += list(c[o:o + n])
        o += n
    sep = I.Basis(atom=np.array(atom, dtype=np.int32), l=np.array(l, dtype=np.int32),
                  nprim=np.array(nprim, dtype=np.int32), exps=np.array(exps), coefs=np.array(coefs))
    m_sp, m_sep = oracle_mod.Molecule(g, sp), oracle_mod.Molecule(g, sep)
    assert m_sp.n_bf == m_sep.n_bf == 15 + 2 + 2
    S1, H1 = m_sp.core_hamiltonian()
    S2, H2 = m_sep.core_hamiltonian()
    assert np.abs(S1 - S2).max() == 0.0 and np.abs(H1 - H2).max() == 0.0
    assert np.allclose(np.diag(S1), 1.0, atol=1e-14)
    # the p functions of an sp shell use the p coefficients: a basis whose sp shells take their s
    # coefficients for p too is a different basis
    same = I.Basis(atom=sp.atom, l=sp.l, nprim=sp.nprim, exps=sp.exps, coefs=sp.coefs, coefs_p=sp.coefs.copy())
    S3, _ = oracle_mod.Molecule(g, same).core_hamiltonian()
    assert np.abs(S3 - S1).max() > 1e-3
    e1 = oracle_mod.scf(m_sp, e_tol=1e-11, d_tol=1e-8)
    e2 = oracle_mod.scf(m_sep, e_tol=1e-11, d_tol=1e-8)
    assert e1.converged and abs(e1.energy - e2.energy) < 1e-12
