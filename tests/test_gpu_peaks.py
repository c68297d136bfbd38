"""The library's roofline microbenchmarks return plausible device rates."""
import pytest

pytestmark = pytest.mark.gpu


def test_measure_peaks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_00033_gb300 import hf
    ctx = hf.Context(0)
    p = hf.measure_peaks(ctx)
    assert p["num_sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    # rates positive and ordered as on every current NVIDIA GPU; FP32 FMA at most 128 lanes per SM per cycle
    assert 0 < p["fp64_fma_gflops"] < p["fp32_fma_gflops"]
    assert 0 < p["red_add_f64_random_gops"] and 0 < p["red_add_f64_coalesced_gops"]
    derived = p["num_sms"] * 128 * 2 * p["sm_max_mhz"] * 1e-3  # 128 FP32 lanes per SM
    assert p["fp32_fma_gflops"] <= 1.05 * derived
