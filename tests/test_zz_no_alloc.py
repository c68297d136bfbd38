"""hf_fock_build_noalloc against hf_fock_build.

The allocation-free entry point serves callers that cannot allocate device
memory during a call (device memory reserved up front or owned by a pool that
forbids cudaMalloc).  It must give the same F, J and K as the regular entry
point, on consecutive calls that share its fixed scratch array, and refuse
systems larger than its stated limit.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1708_00033_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_00033_gb300 import hf
    return hf.Context(0)


def _sym_density(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n // 5))
    return 0.2 * (G @ G.T)


@pytest.mark.parametrize("tau", [0.0, 1e-10])
def test_noalloc_matches_regular_build_twice(ctx, tau):
    import torch
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=tau)
    N = s.n_bf
    for call, seed in enumerate((1, 2)):
        P = torch.from_numpy(_sym_density(N, seed)).cuda()
        ref = s.fock_build(P, want_J=True, want_K=True, energy=False)
        F = torch.full_like(P, float("nan"))
        J = torch.full_like(P, float("nan"))
        K = torch.full_like(P, float("nan"))
        hf.fock_build_noalloc(s, P, F, J, K)
        torch.cuda.synchronize()
        for name, got, want in (("F", F, ref["F"]), ("J", J, ref["J"]), ("K", K, ref["K"])):
            err = float((got - want).abs().max())
            assert err <= TOL, (call, name, err)


def test_noalloc_rejects_systems_over_the_limit(ctx):
    import torch
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(21, I.CONFIG_SINGLE_BUILD, 5)  # 525 basis functions > 512
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10)
    assert s.n_bf > 512
    P = torch.eye(s.n_bf, dtype=torch.float64, device="cuda")
    F = torch.empty_like(P)
    with pytest.raises(hf.HFError) as e:
        hf.fock_build_noalloc(s, P, F)
    assert e.value.code == hf.HF_E_INVALID
