"""Mixed precision: quartets with Q_ij Q_kl < 1e-4 evaluated in FP32 (FP64
accumulation), the rest in FP64, on the first 16 waters of the 256-water
cluster, against oracle values written by tests/golden/make_mixed16_golden.py.

Tolerances: the mixed energy within 1e-6 Eh of the FP64 oracle (the stated
mixed-precision target); sampled F elements within 1e-5 (FP32 rounding of
integrals below 1e-4 summed over ~1e7 quartets); the FP64 path within 1e-10.
"""
import json
import os

import numpy as np
import pytest

from paper_1708_00033_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mixed16_oracle.json")


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1708_00033_gb300 import hf
    ref = json.load(open(GOLDEN))
    geom = I.subset_waters(I.water_cluster(256, I.CONFIG_MIXED), 16)
    basis = I.synthetic_basis(geom)
    mol = oracle.Molecule(geom, basis)
    S, H = mol.core_hamiltonian()
    P = oracle.density_from_orbitals(oracle.orthonormalise(I.random_orbitals(mol.n_bf, 80, I.CONFIG_MIXED, 0), S))
    return hf.Context(0), geom, basis, P, ref


def _sampled(M, pairs):
    return np.array([M[a, b] for a, b in pairs])


def test_fp64_matches_oracle(setup):
    from paper_1708_00033_gb300 import hf
    ctx, geom, basis, P, ref = setup
    s = hf.System(ctx, geom, basis, schwarz_tau=ref["tau"])
    out = s.fock_build(P, want_J=True, want_K=True, stats=True)
    assert abs(out["stats"]["quartets_fp64"] - ref["quartets"]) <= 2
    assert np.abs(_sampled(out["F"], ref["pairs"]) - np.array(ref["F"])).max() <= 1e-10
    assert abs(out["E_elec"] - ref["E_elec"]) <= 1e-9


def test_mixed_energy_within_1e6(setup):
    from paper_1708_00033_gb300 import hf
    ctx, geom, basis, P, ref = setup
    s = hf.System(ctx, geom, basis, schwarz_tau=ref["tau"], fp32_cutoff=1e-4)
    out = s.fock_build(P, want_J=True, want_K=True, stats=True)
    st = out["stats"]
    assert st["quartets_fp32"] > 0.5 * (st["quartets_fp32"] + st["quartets_fp64"])
    dE = abs(out["E_elec"] - ref["E_elec"])
    dF = np.abs(_sampled(out["F"], ref["pairs"]) - np.array(ref["F"])).max()
    assert dE <= 1e-6, dE
    assert dF <= 1e-5, dF


def test_mixed_cutoff_zero_is_fp64(setup):
    from paper_1708_00033_gb300 import hf
    ctx, geom, basis, P, ref = setup
    s = hf.System(ctx, geom, basis, schwarz_tau=ref["tau"], fp32_cutoff=0.0)
    out = s.fock_build(P, stats=True)
    assert out["stats"]["quartets_fp32"] == 0
