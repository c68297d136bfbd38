"""hf_fock_build_noalloc against hf_fock_build.

The allocation-free entry point serves callers that cannot allocate device
memory during a call (device memory reserved up front or owned by a pool that
forbids cudaMalloc).  It must give the same F, J and K as the regular entry
point, on consecutive calls that share its fixed scratch array, for FP64 and
mixed-precision systems; it must leave the device's free memory unchanged;
it must reject an invalid density without touching its outputs and stay
usable afterwards; and it must refuse systems larger than its stated limit.
This file is collected last.
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


@pytest.mark.parametrize("tau,cutoff", [(0.0, 0.0), (1e-10, 0.0), (1e-10, 1e-4)])
def test_noalloc_matches_regular_build_twice(ctx, tau, cutoff):
    """Two calls in a row against hf_fock_build on the same system (for a mixed system both evaluate the
    same quartets in FP32), and no change of the device's free memory across the calls."""
    import torch
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(4, I.CONFIG_SINGLE_BUILD)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=tau, fp32_cutoff=cutoff)
    if cutoff > 0:
        assert s.info["quartets_fp32"] > 0
    N = s.n_bf
    Ps = [torch.from_numpy(_sym_density(N, seed)).cuda() for seed in (1, 2)]
    refs = [s.fock_build(P, want_J=True, want_K=True, energy=False) for P in Ps]
    outs = [tuple(torch.full_like(Ps[0], float("nan")) for _ in range(3)) for _ in Ps]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for P, (F, J, K) in zip(Ps, outs):
        hf.fock_build_noalloc(s, P, F, J, K)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    tol = TOL if cutoff == 0 else 1e-12 * max(1.0, float(refs[0]["F"].abs().max()))
    for call, (ref, (F, J, K)) in enumerate(zip(refs, outs)):
        for name, got, want in (("F", F, ref["F"]), ("J", J, ref["J"]), ("K", K, ref["K"])):
            err = float((got - want).abs().max())
            assert err <= max(tol, TOL), (call, name, err)


def test_noalloc_rejects_invalid_density_then_recovers(ctx):
    import torch
    from paper_1708_00033_gb300 import hf
    geom = I.water_cluster(2, I.CONFIG_SINGLE_BUILD, 3)
    basis = I.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=1e-10)
    N = s.n_bf
    P = torch.from_numpy(_sym_density(N, 5)).cuda()
    bad = P.clone()
    bad[1, 2] += 0.5  # not symmetric
    F = torch.full_like(P, 3.0)
    with pytest.raises(hf.HFError) as e:
        hf.fock_build_noalloc(s, bad, F)
    assert e.value.code == hf.HF_E_INVALID
    assert bool((F == 3.0).all())
    hf.fock_build_noalloc(s, P, F)
    ref = s.fock_build(P, energy=False)
    assert float((F - ref["F"]).abs().max()) <= TOL


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
