"""Seeded synthetic inputs for the direct-SCF Fock build.

This module only draws and lays out inputs: water-cluster geometries, the
synthetic even-tempered Cartesian basis (raw exponents and contraction
coefficients) and Gaussian random orbital matrices.  It holds none of the
method's arithmetic (no normalisation, no integrals, no densities), so the
CPU oracle and the CUDA path can both consume it without sharing any of the
computation they are compared on.

Geometry recipe (the project's own definition of a "3.0 A jittered cubic grid"
cluster of rigid waters):
  * n waters fill the first n points of a ceil(n^(1/3))^3 grid with 3.0 A
    spacing, x index fastest;
  * each O sits at its grid point plus a U(-0.3, 0.3) A jitter per axis;
  * each molecule gets a uniformly random orientation (Shoemake's
    quaternion construction);
  * O-H = 0.96 A and H-O-H = 104.5 deg in the molecule frame;
  * a molecule that would put any of its atoms within 1.6 A of an atom of an
    earlier molecule is redrawn.
Seeds are the pair (config id, molecule index) fed to numpy's SeedSequence,
driving one PCG64 stream per cluster.

Basis (per element; every shell is a 3-primitive contraction with exponents
alpha*{1, 3, 9} and coefficients {0.4, 0.4, 0.2} that multiply *normalised*
primitives):
  O: s(0.2) s(2.0) s(20.0) p(0.3) p(3.0) d(0.8)   -> 15 Cartesian functions
  H: s(0.15) s(1.5) p(0.5)                        ->  5 Cartesian functions
Cartesian component order: p = x, y, z; d = xx, xy, xz, yy, yz, zz.
Units: bohr; 1 bohr = 0.529177210903 A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BOHR_IN_ANGSTROM = 0.529177210903
ANGSTROM_IN_BOHR = 1.0 / BOHR_IN_ANGSTROM

OH_BOND_A = 0.96
HOH_ANGLE_DEG = 104.5
GRID_SPACING_A = 3.0
JITTER_A = 0.3
MIN_CONTACT_A = 1.6

PRIM_SCALE = (1.0, 3.0, 9.0)
PRIM_COEF = (0.4, 0.4, 0.2)

# (l, base exponent) per element, in shell order.
SHELLS_BY_Z = {
    8: ((0, 0.2), (0, 2.0), (0, 20.0), (1, 0.3), (1, 3.0), (2, 0.8)),
    1: ((0, 0.15), (0, 1.5), (1, 0.5)),
}

NCART = (1, 3, 6)

# Configuration ids used as the first seed word.
CONFIG_SINGLE_BUILD = 1     # 4 waters, no screening
CONFIG_SCF = 2              # 64 waters, SCF
CONFIG_MIXED = 3            # 256 waters, mixed precision
CONFIG_BATCH = 4            # 512 molecules of 1..16 waters
CONFIG_GUESS_TRAIN = 5      # learned-guess training clusters
CONFIG_GUESS_EVAL = 6       # learned-guess held-out clusters

# Thresholds of the benchmarked workloads: Schwarz screening of shell quartets and the primitive-pair
# threshold (a primitive quartet is skipped when the product of its two primitive-pair bounds is below it).
BENCH_SCHWARZ_TAU = 1e-10
BENCH_PRIM_TAU = 1e-14


@dataclass
class Geometry:
    Z: np.ndarray        # int32 [n_atoms]
    xyz: np.ndarray      # float64 [n_atoms, 3], bohr

    @property
    def n_atoms(self) -> int:
        return int(self.Z.shape[0])


@dataclass
class Basis:
    atom: np.ndarray     # int32 [n_shells] atom index of each shell
    l: np.ndarray        # int32 [n_shells] angular momentum 0..2
    nprim: np.ndarray    # int32 [n_shells]
    exps: np.ndarray     # float64 [sum nprim] primitive exponents
    coefs: np.ndarray    # float64 [sum nprim] coefficients on normalised primitives (s part of sp shells)
    coefs_p: np.ndarray | None = None  # float64 [sum nprim] p coefficients of sp shells (l = -1), else unused

    @property
    def n_shells(self) -> int:
        return int(self.l.shape[0])

    @property
    def n_bf(self) -> int:
        return int(sum(NCART[int(x)] for x in self.l))

    def prim_offsets(self) -> np.ndarray:
        off = np.zeros(self.n_shells + 1, dtype=np.int64)
        np.cumsum(self.nprim, out=off[1:])
        return off

    def bf_offsets(self) -> np.ndarray:
        off = np.zeros(self.n_shells + 1, dtype=np.int64)
        np.cumsum([NCART[int(x)] for x in self.l], out=off[1:])
        return off


def cluster_rng(config_id: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(config_id), int(index)])))


def _icbrt_ceil(n: int) -> int:
    s = 1
    while s * s * s < n:
        s += 1
    return s


def _shoemake_rotation(u: np.ndarray) -> np.ndarray:
    u1, u2, u3 = float(u[0]), float(u[1]), float(u[2])
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _water_frame_angstrom() -> np.ndarray:
    h = math.radians(HOH_ANGLE_DEG) / 2.0
    return np.array([
        [0.0, 0.0, 0.0],
        [OH_BOND_A * math.sin(h), 0.0, OH_BOND_A * math.cos(h)],
        [-OH_BOND_A * math.sin(h), 0.0, OH_BOND_A * math.cos(h)],
    ])


def water_cluster(n_waters: int, config_id: int, index: int = 0, rng: np.random.Generator | None = None) -> Geometry:
    """Seeded cluster of ``n_waters`` rigid waters (atoms O, H, H per water)."""
    if n_waters < 1:
        raise ValueError("n_waters must be >= 1")
    if rng is None:
        rng = cluster_rng(config_id, index)
    side = _icbrt_ceil(n_waters)
    frame = _water_frame_angstrom()
    placed: list[np.ndarray] = []
    for w in range(n_waters):
        g = np.array([w % side, (w // side) % side, w // (side * side)], dtype=np.float64) * GRID_SPACING_A
        for _attempt in range(10000):
            jit = rng.uniform(-JITTER_A, JITTER_A, size=3)
            rot = _shoemake_rotation(rng.uniform(0.0, 1.0, size=3))
            mol = (frame @ rot.T) + (g + jit)
            if placed:
                prev = np.concatenate(placed, axis=0)
                d = np.sqrt(((mol[:, None, :] - prev[None, :, :]) ** 2).sum(-1))
                if d.min() < MIN_CONTACT_A:
                    continue
            break
        else:  # pragma: no cover - geometric impossibility at this spacing
            raise RuntimeError("could not place water without contacts")
        placed.append(mol)
    xyz = np.concatenate(placed, axis=0) * ANGSTROM_IN_BOHR
    Z = np.tile(np.array([8, 1, 1], dtype=np.int32), n_waters)
    return Geometry(Z=Z, xyz=np.ascontiguousarray(xyz, dtype=np.float64))


def subset_waters(geom: Geometry, n_waters: int) -> Geometry:
    """First ``n_waters`` molecules of a water cluster (atoms are O,H,H per water)."""
    n = 3 * n_waters
    return Geometry(Z=geom.Z[:n].copy(), xyz=geom.xyz[:n].copy())


def batch_cluster_sizes(n_mol: int, config_id: int = CONFIG_BATCH, lo: int = 1, hi: int = 16) -> list[int]:
    """Sizes U{lo..hi} of the clusters in a batch; drawn from each cluster's own stream."""
    return [int(cluster_rng(config_id, m).integers(lo, hi + 1)) for m in range(n_mol)]


def batch_cluster(config_id: int, m: int, lo: int = 1, hi: int = 16) -> Geometry:
    rng = cluster_rng(config_id, m)
    n = int(rng.integers(lo, hi + 1))
    return water_cluster(n, config_id, m, rng=rng)


def synthetic_basis(geom: Geometry) -> Basis:
    atom, l, nprim, exps, coefs = [], [], [], [], []
    for a, z in enumerate(geom.Z.tolist()):
        if z not in SHELLS_BY_Z:
            raise ValueError(f"no basis for Z={z}")
        for (lq, base) in SHELLS_BY_Z[z]:
            atom.append(a)
            l.append(lq)
            nprim.append(len(PRIM_SCALE))
            exps.extend(base * s for s in PRIM_SCALE)
            coefs.extend(PRIM_COEF)
    return Basis(atom=np.array(atom, dtype=np.int32), l=np.array(l, dtype=np.int32),
                 nprim=np.array(nprim, dtype=np.int32), exps=np.array(exps, dtype=np.float64),
                 coefs=np.array(coefs, dtype=np.float64))


# Split-valence synthetic basis with sp (L) shells (the shape of 6-31G(d): core s, two sp valence shells,
# polarisation d on O; two s on H): per shell (l, base exponent, s coefficients, p coefficients), the
# primitive exponents being base * PRIM_SCALE[:n] for n coefficients.  l = -1 is an sp shell.
SP_SHELLS_BY_Z = {
    8: [(0, 20.0, (0.4, 0.4, 0.2), None),
        (-1, 1.2, (-0.1, 0.5, 0.6), (0.3, 0.5, 0.3)),
        (-1, 0.25, (1.0,), (1.0,)),
        (2, 0.8, (1.0,), None)],
    1: [(0, 1.5, (0.4, 0.4, 0.2), None),
        (0, 0.15, (1.0,), None)],
}


def synthetic_sp_basis(geom: Geometry) -> Basis:
    """The split-valence synthetic basis: 15 functions on O (s, sp, sp, d), 2 on H (s, s)."""
    atom, l, nprim, exps, coefs, coefs_p = [], [], [], [], [], []
    for a, z in enumerate(geom.Z.tolist()):
        if z not in SP_SHELLS_BY_Z:
            raise ValueError(f"no basis for Z={z}")
        for (lq, base, cs, cp) in SP_SHELLS_BY_Z[z]:
            atom.append(a)
            l.append(lq)
            nprim.append(len(cs))
            exps.extend(base * s for s in PRIM_SCALE[:len(cs)])
            coefs.extend(cs)
            coefs_p.extend(cp if cp is not None else (0.0,) * len(cs))
    return Basis(atom=np.array(atom, dtype=np.int32), l=np.array(l, dtype=np.int32),
                 nprim=np.array(nprim, dtype=np.int32), exps=np.array(exps, dtype=np.float64),
                 coefs=np.array(coefs, dtype=np.float64), coefs_p=np.array(coefs_p, dtype=np.float64))


def random_orbitals(n_bf: int, n_occ: int, config_id: int, index: int = 0) -> np.ndarray:
    """G ~ N(0,1), shape [n_bf, n_occ]; orthonormalisation is left to the caller."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(config_id), int(index), 1])))
    return rng.standard_normal((n_bf, n_occ))


def guess_init_weights(seed: int = 0) -> np.ndarray:
    """Seeded initial weights of the learned-guess MLP (float32, in the library's layout W1[256][16], b1,
    W2[256][256], b2, W3[325][256], b3): He-uniform matrices (the output layer scaled by 0.1), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((16, 256), (256, 256), (256, 325)):
        lim = math.sqrt(6.0 / fan_in) * (1.0 if fan_out != 325 else 0.1)
        parts.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32).ravel())
        parts.append(np.zeros(fan_out, dtype=np.float32))
    return np.concatenate(parts)


def n_electrons(geom: Geometry) -> int:
    return int(geom.Z.sum())


# Hehre-Stewart-Pople STO-3G hydrogen 1s (zeta = 1.24) as tabulated by
# Szabo & Ostlund, used only for the H2 textbook check.
STO3G_H_EXPS = (3.42525091, 0.62391373, 0.16885540)
STO3G_H_COEFS = (0.15432897, 0.53532814, 0.44463454)


def h2_sto3g(r_bohr: float = 1.4) -> tuple[Geometry, Basis]:
    geom = Geometry(Z=np.array([1, 1], dtype=np.int32), xyz=np.array([[0.0, 0.0, 0.0], [0.0, 0.0, r_bohr]]))
    basis = Basis(atom=np.array([0, 1], dtype=np.int32), l=np.array([0, 0], dtype=np.int32),
                  nprim=np.array([3, 3], dtype=np.int32), exps=np.array(STO3G_H_EXPS * 2),
                  coefs=np.array(STO3G_H_COEFS * 2))
    return geom, basis
