"""Writes tests/golden/mixed16_oracle.json with the CPU oracle only.

Workload: the first 16 waters of the 256-water mixed-precision cluster
(seed (3, 0)), 400 basis functions, random S-orthonormal density with 80
occupied orbitals (seed (3, 0)), Schwarz screening at 1e-10.  Stored: the
oracle's electronic energy, J/K/F on a fixed sample of elements, and the
screened quartet count.  Run:  python tests/golden/make_mixed16_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1708_00033_gb300 import inputs as I  # noqa: E402

TAU = 1e-10


def workload():
    geom = I.subset_waters(I.water_cluster(256, I.CONFIG_MIXED), 16)
    basis = I.synthetic_basis(geom)
    mol = oracle.Molecule(geom, basis)
    S, H = mol.core_hamiltonian()
    C = oracle.orthonormalise(I.random_orbitals(mol.n_bf, 80, I.CONFIG_MIXED, 0), S)
    return geom, basis, mol, S, H, oracle.density_from_orbitals(C)


def sample_indices(n, k=400, seed=7):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, size=(k, 2))
    return [(int(a), int(b)) for a, b in idx] + [(i, i) for i in range(0, n, 7)]


def main():
    geom, basis, mol, S, H, P = workload()
    J, K = mol.jk_unique(P, TAU)
    F = oracle.fock_from_jk(H, J, K)
    E = oracle.electronic_energy(P, H, F)
    pairs = sample_indices(mol.n_bf)
    out = {
        "workload": "first 16 waters of the 256-water cluster seed (3,0); random-C density n_occ=80 seed (3,0); tau=1e-10",
        "n_bf": mol.n_bf, "tau": TAU, "E_elec": E, "quartets": mol.last_quartets,
        "pairs": pairs,
        "F": [float(F[a, b]) for a, b in pairs], "J": [float(J[a, b]) for a, b in pairs],
        "K": [float(K[a, b]) for a, b in pairs],
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "mixed16_oracle.json"), "w") as fh:
        json.dump(out, fh)
    print("E_elec", E, "quartets", mol.last_quartets)


if __name__ == "__main__":
    main()
