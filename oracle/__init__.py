"""CPU FP64 oracle for the direct-SCF Fock build.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  It
shares no code with the CUDA library: its integrals use the
McMurchie-Davidson Hermite expansion (``hf_oracle.c``), the library's the
Obara-Saika / Head-Gordon-Pople recurrences.

What each function follows:
  * ``one_electron``   S, T, V and E_nn of Section 3 (the O(N^2) part);
  * ``jk_literal``     J and K by their definitions over all ordered indices;
  * ``jk_unique``      Algorithm 1's unique shell quartets + Eq. 1a-1f;
  * ``jk_elements``    single J/K elements by definition (large systems);
  * ``jk_shell_blocks`` whole shell blocks of J/K by definition (large systems);
  * ``fock``           F = H + J - K/2, E = 1/2 tr P(H+F) + E_nn;
  * ``scf``            the SCF cycle of Section 3 (symmetric orthogonalisation,
                       core-Hamiltonian guess, diagonalise, new density, stop on
                       RMS density change), with Pulay DIIS added.
Parity pins live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle's C source with gcc (-O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    lib.or_create.restype = ctypes.c_void_p
    lib.or_create.argtypes = [ctypes.c_int, _ip, _dp, ctypes.c_int, _ip, _ip, _ip, _dp, _dp]
    lib.or_destroy.argtypes = [ctypes.c_void_p]
    lib.or_nbf.restype = ctypes.c_int
    lib.or_nbf.argtypes = [ctypes.c_void_p]
    lib.or_shell_info.argtypes = [ctypes.c_void_p, _ip, _ip]
    lib.or_boys.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
    lib.or_nuclear_repulsion.restype = ctypes.c_double
    lib.or_nuclear_repulsion.argtypes = [ctypes.c_void_p]
    lib.or_one_electron.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    lib.or_eri_shell_quartet.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
    lib.or_eri_primitive.restype = ctypes.c_double
    lib.or_eri_primitive.argtypes = [_ip, ctypes.c_double, _dp] * 4
    lib.or_schwarz.argtypes = [ctypes.c_void_p, _dp]
    lib.or_one_electron_primitive.argtypes = [_ip, ctypes.c_double, _dp, _ip, ctypes.c_double, _dp, ctypes.c_double, _dp, _dp]
    lib.or_packed_size.restype = ctypes.c_int64
    lib.or_packed_size.argtypes = [ctypes.c_void_p]
    lib.or_eri_packed.argtypes = [ctypes.c_void_p, _dp]
    lib.or_jk_literal.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
    lib.or_jk_unique.restype = ctypes.c_int64
    lib.or_jk_unique.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp, _dp, _dp]
    lib.or_jk_unique_sample.restype = ctypes.c_int64
    lib.or_jk_unique_sample.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp, ctypes.c_int64, ctypes.c_int64, _dp, _dp, ctypes.POINTER(ctypes.c_int64)]
    lib.or_jk_elements.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp, ctypes.c_int, _ip, _ip, _dp, _dp]
    lib.or_jk_unique_rows.restype = ctypes.c_int64
    lib.or_jk_unique_rows.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int64), _dp, _dp, _dp]
    lib.or_jk_shell_blocks.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, _dp, ctypes.c_int, _ip, _ip, _dp, _dp]
    lib.or_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    return a.ctypes.data_as(_ip)


def num_threads() -> int:
    return int(_load().or_num_threads())


def boys(mmax: int, T: float) -> np.ndarray:
    out = np.zeros(mmax + 1)
    _load().or_boys(int(mmax), float(T), _d(out))
    return out


def eri_primitive(pa, a, A, pb, b, B, pc, c, C, pd, d, D) -> float:
    """Unnormalised primitive Cartesian ERI [ab|cd] (powers, exponent, centre per index)."""
    arrays, cargs = [], []
    for pw, ex, ctr in ((pa, a, A), (pb, b, B), (pc, c, C), (pd, d, D)):
        pwa = np.ascontiguousarray(pw, dtype=np.int32)
        ca = np.ascontiguousarray(ctr, dtype=np.float64)
        arrays += [pwa, ca]
        cargs += [_i(pwa), float(ex), _d(ca)]
    return float(_load().or_eri_primitive(*cargs))


def one_electron_primitive(pa, a, A, pb, b, B, Zc, C):
    """Unnormalised primitive (S, T, V_C) for one pair and one point charge Zc at C."""
    pa_, pb_ = np.ascontiguousarray(pa, dtype=np.int32), np.ascontiguousarray(pb, dtype=np.int32)
    A_, B_, C_ = (np.ascontiguousarray(x, dtype=np.float64) for x in (A, B, C))
    out = np.zeros(3)
    _load().or_one_electron_primitive(_i(pa_), float(a), _d(A_), _i(pb_), float(b), _d(B_), float(Zc), _d(C_), _d(out))
    return out


def _split_sp(basis):
    """Shell lists with every sp (L) shell (l = -1) written as its s shell (coefficients coefs) followed by
    its p shell (coefficients coefs_p), both with the sp shell's exponents: an sp shell is by definition
    those two shells sharing exponents, with functions s, x, y, z."""
    l_in = np.asarray(basis.l)
    if not np.any(l_in == -1):
        return basis.atom, basis.l, basis.nprim, basis.exps, basis.coefs
    atom, l, nprim, exps, coefs = [], [], [], [], []
    o = 0
    for s_ in range(l_in.size):
        n = int(basis.nprim[s_])
        e = list(basis.exps[o:o + n])
        if l_in[s_] == -1:
            for lq, c in ((0, basis.coefs), (1, basis.coefs_p)):
                atom.append(int(basis.atom[s_]))
                l.append(lq)
                nprim.append(n)
                exps += e
                coefs += list(c[o:o + n])
        else:
            atom.append(int(basis.atom[s_]))
            l.append(int(l_in[s_]))
            nprim.append(n)
            exps += e
            coefs += list(basis.coefs[o:o + n])
        o += n
    return atom, l, nprim, exps, coefs


class Molecule:
    """A geometry + basis handle on the oracle side (sp shells are split into s and p shells)."""

    def __init__(self, geom, basis):
        lib = _load()
        self.Z = np.ascontiguousarray(geom.Z, dtype=np.int32)
        self.xyz = np.ascontiguousarray(geom.xyz, dtype=np.float64)
        atom, l, nprim, exps, coefs = _split_sp(basis)
        self._atom = np.ascontiguousarray(atom, dtype=np.int32)
        self._l = np.ascontiguousarray(l, dtype=np.int32)
        self._nprim = np.ascontiguousarray(nprim, dtype=np.int32)
        self._exps = np.ascontiguousarray(exps, dtype=np.float64)
        self._coefs = np.ascontiguousarray(coefs, dtype=np.float64)
        self.n_shells = int(self._l.shape[0])
        h = lib.or_create(int(self.Z.shape[0]), _i(self.Z), _d(self.xyz), self.n_shells, _i(self._atom),
                          _i(self._l), _i(self._nprim), _d(self._exps), _d(self._coefs))
        if not h:
            raise ValueError("oracle rejected the basis (l > 2 or bad primitive count)")
        self._h = ctypes.c_void_p(h)
        self.n_bf = int(lib.or_nbf(self._h))
        self.bf0 = np.zeros(self.n_shells, dtype=np.int32)
        self.ncomp = np.zeros(self.n_shells, dtype=np.int32)
        lib.or_shell_info(self._h, _i(self.bf0), _i(self.ncomp))
        self.n_electrons = int(self.Z.sum())
        self._Q = None

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None and _lib is not None:
                _lib.or_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def nuclear_repulsion(self) -> float:
        return float(_load().or_nuclear_repulsion(self._h))

    def one_electron(self):
        N = self.n_bf
        S, T, V = np.zeros((N, N)), np.zeros((N, N)), np.zeros((N, N))
        _load().or_one_electron(self._h, _d(S), _d(T), _d(V))
        return S, T, V

    def core_hamiltonian(self):
        S, T, V = self.one_electron()
        return S, T + V

    def eri_shell_quartet(self, i, j, k, l) -> np.ndarray:
        out = np.zeros((int(self.ncomp[i]), int(self.ncomp[j]), int(self.ncomp[k]), int(self.ncomp[l])))
        _load().or_eri_shell_quartet(self._h, int(i), int(j), int(k), int(l), _d(out))
        return out

    def schwarz(self) -> np.ndarray:
        if self._Q is None:
            Q = np.zeros((self.n_shells, self.n_shells))
            _load().or_schwarz(self._h, _d(Q))
            self._Q = Q
        return self._Q

    def eri_packed(self) -> np.ndarray:
        n = int(_load().or_packed_size(self._h))
        if n > 60_000_000:
            raise MemoryError("packed ERI table too large for the literal path")
        out = np.zeros(n)
        _load().or_eri_packed(self._h, _d(out))
        return out

    def eri_full(self) -> np.ndarray:
        """Full N^4 tensor (tiny systems only), expanded from the packed table."""
        N = self.n_bf
        pk = self.eri_packed()
        idx = np.arange(N)
        a, b = np.meshgrid(idx, idx, indexing="ij")
        p2 = np.where(a >= b, a * (a + 1) // 2 + b, b * (b + 1) // 2 + a)
        x, y = np.meshgrid(p2.ravel(), p2.ravel(), indexing="ij")
        p4 = np.where(x >= y, x * (x + 1) // 2 + y, y * (y + 1) // 2 + x)
        return pk[p4].reshape(N, N, N, N)

    def jk_literal(self, P: np.ndarray, eri_packed: np.ndarray | None = None):
        N = self.n_bf
        if eri_packed is None:
            eri_packed = self.eri_packed()
        P = np.ascontiguousarray(P, dtype=np.float64)
        J, K = np.zeros((N, N)), np.zeros((N, N))
        _load().or_jk_literal(N, _d(eri_packed), _d(P), _d(J), _d(K))
        return J, K

    def jk_unique(self, P: np.ndarray, tau: float = 0.0):
        N = self.n_bf
        P = np.ascontiguousarray(P, dtype=np.float64)
        J, K = np.zeros((N, N)), np.zeros((N, N))
        Q = self.schwarz() if tau > 0 else np.zeros((1, 1))
        n = _load().or_jk_unique(self._h, _d(P), float(tau), _d(np.ascontiguousarray(Q)), _d(J), _d(K))
        self.last_quartets = int(n)
        return J, K

    def jk_unique_sample(self, P: np.ndarray, tau: float, stride: int, offset: int = 0):
        """Unique-quartet digestion over every stride-th bra pair; returns
        (quartets evaluated, unscreened quartets the sampled rows span)."""
        N = self.n_bf
        P = np.ascontiguousarray(P, dtype=np.float64)
        J, K = np.zeros((N, N)), np.zeros((N, N))
        Q = self.schwarz() if tau > 0 else np.zeros((1, 1))
        u = ctypes.c_int64(0)
        n = _load().or_jk_unique_sample(self._h, _d(P), float(tau), _d(np.ascontiguousarray(Q)), int(stride),
                                        int(offset), _d(J), _d(K), ctypes.byref(u))
        return int(n), int(u.value)

    def jk_unique_rows(self, P: np.ndarray, tau: float, rows):
        """Unique-quartet digestion over the given bra pairs ij (rows of Algorithm 1's outer loop); returns
        (quartets evaluated, seconds the threads spent in the rows summed over threads).  J and K of the
        partial sum are discarded."""
        N = self.n_bf
        P = np.ascontiguousarray(P, dtype=np.float64)
        J, K = np.zeros((N, N)), np.zeros((N, N))
        Q = self.schwarz() if tau > 0 else np.zeros((1, 1))
        r = np.ascontiguousarray(rows, dtype=np.int64)
        busy = ctypes.c_double(0.0)
        n = _load().or_jk_unique_rows(self._h, _d(P), float(tau), _d(np.ascontiguousarray(Q)), int(r.size),
                                      r.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _d(J), _d(K),
                                      ctypes.byref(busy))
        return int(n), float(busy.value)

    def jk_elements(self, P: np.ndarray, pairs, tau: float = 0.0):
        P = np.ascontiguousarray(P, dtype=np.float64)
        mu = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
        nu = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
        Jel, Kel = np.zeros(len(pairs)), np.zeros(len(pairs))
        Q = self.schwarz() if tau > 0 else np.zeros((1, 1))
        _load().or_jk_elements(self._h, _d(P), float(tau), _d(np.ascontiguousarray(Q)), len(pairs), _i(mu), _i(nu),
                               _d(Jel), _d(Kel))
        return Jel, Kel

    def jk_shell_blocks(self, P: np.ndarray, blocks, tau: float = 0.0):
        """Whole (I, J) shell blocks of J and K by definition (list of (ncomp_I x ncomp_J) arrays each)."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        Il = np.ascontiguousarray([b[0] for b in blocks], dtype=np.int32)
        Jl = np.ascontiguousarray([b[1] for b in blocks], dtype=np.int32)
        sizes = [int(self.ncomp[i]) * int(self.ncomp[j]) for i, j in blocks]
        Jo, Ko = np.zeros(sum(sizes)), np.zeros(sum(sizes))
        Q = self.schwarz() if tau > 0 else np.zeros((1, 1))
        _load().or_jk_shell_blocks(self._h, _d(P), float(tau), _d(np.ascontiguousarray(Q)), len(blocks), _i(Il), _i(Jl),
                                   _d(Jo), _d(Ko))
        outJ, outK, o = [], [], 0
        for (i, j), n in zip(blocks, sizes):
            shp = (int(self.ncomp[i]), int(self.ncomp[j]))
            outJ.append(Jo[o:o + n].reshape(shp))
            outK.append(Ko[o:o + n].reshape(shp))
            o += n
        return outJ, outK


def fock_from_jk(H, J, K):
    """F = H + J - K/2 for a closed-shell total density."""
    return H + J - 0.5 * K


def electronic_energy(P, H, F) -> float:
    """E_elec = 1/2 sum P_mu nu (H_mu nu + F_mu nu)."""
    return 0.5 * float(np.sum(P * (H + F)))


def density_from_orbitals(C_occ: np.ndarray) -> np.ndarray:
    """Total closed-shell density P = 2 C_occ C_occ^T."""
    return 2.0 * C_occ @ C_occ.T


def orthonormalise(G: np.ndarray, S: np.ndarray) -> np.ndarray:
    """C = G L^-T with L L^T = G^T S G, so that C^T S C = 1."""
    L = np.linalg.cholesky(G.T @ S @ G)
    return np.linalg.solve(L, G.T).T


@dataclass
class SCFResult:
    energy: float
    iterations: int
    converged: bool
    P: np.ndarray
    eps: np.ndarray
    history: list = field(default_factory=list)


def scf(mol: Molecule, n_occ: int | None = None, tau: float = 0.0, e_tol: float = 1e-9, d_tol: float = 1e-6,
        max_iter: int = 100, diis_size: int = 8, P_guess: np.ndarray | None = None, fock_builder=None) -> SCFResult:
    """Closed-shell SCF of Section 3.

    Symmetric (Lowdin) orthogonalisation X = S^-1/2 (canonical when an S
    eigenvalue is below 1e-8), core-Hamiltonian guess, then repeat: build F(P),
    Pulay-extrapolate F from the last ``diis_size`` error vectors FPS - SPF,
    diagonalise X^T F X, occupy the lowest ``n_occ`` orbitals, and stop when
    |dE| < e_tol and the RMS density change < d_tol.
    """
    if n_occ is None:
        n_occ = mol.n_electrons // 2
    S, H = mol.core_hamiltonian()
    E_nn = mol.nuclear_repulsion()
    s, U = np.linalg.eigh(S)
    keep = s > 1e-8
    X = U[:, keep] / np.sqrt(s[keep])
    if keep.all():
        X = X @ U.T  # symmetric orthogonalisation

    def diag(F):
        e, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
        return e, density_from_orbitals(C[:, :n_occ])

    if P_guess is None:
        eps, P = diag(H)
    else:
        P = np.array(P_guess, dtype=np.float64)
        eps = np.zeros(0)
    if fock_builder is None:
        def fock_builder(P_):
            J, K = mol.jk_unique(P_, tau)
            return fock_from_jk(H, J, K)
    E_old = None
    fs, es, hist = [], [], []
    for it in range(1, max_iter + 1):
        F = fock_builder(P)
        E = electronic_energy(P, H, F) + E_nn
        err = F @ P @ S - S @ P @ F
        fs.append(F)
        es.append(err)
        if len(fs) > diis_size:
            fs.pop(0)
            es.pop(0)
        if len(fs) >= 2:
            m = len(fs)
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            for a in range(m):
                for b in range(m):
                    B[a, b] = float(np.sum(es[a] * es[b]))
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            try:
                coef = np.linalg.solve(B, rhs)[:m]
                F_use = sum(c * f for c, f in zip(coef, fs))
            except np.linalg.LinAlgError:
                F_use = F
        else:
            F_use = F
        eps, P_new = diag(F_use)
        dP = float(np.sqrt(np.mean((P_new - P) ** 2)))
        hist.append((E, dP))
        if E_old is not None and abs(E - E_old) < e_tol and dP < d_tol:
            return SCFResult(E, it, True, P, eps, hist)
        E_old = E
        P = P_new
    return SCFResult(E, max_iter, False, P, eps, hist)
