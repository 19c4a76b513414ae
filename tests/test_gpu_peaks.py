"""The arithmetic-throughput microbenchmarks behind the walk's roofline give
plausible figures: FP32 FMA within a factor of the SM count x 128 lanes x 2 flops
x clock, rsqrt below the FMA rate, FP64 far below FP32."""
import pytest

pytestmark = pytest.mark.gpu


def test_measure_peaks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0709_3331_gb300 import build as b
    b.build()
    from paper_0709_3331_gb300.ucp import measure_peaks
    p = measure_peaks()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = nsm * 128 * 2 * 2.1e9 / 1e12     # TFLOP/s at a 2.1 GHz upper clock
    assert 0.2 * nominal < p["fp32_fma_tflops"] < 1.05 * nominal
    assert p["fp32x2_fma_tflops"] > 0.5 * p["fp32_fma_tflops"]
    assert 0 < p["rsqrt_gops"] * 1e-3 < p["fp32_fma_tflops"] / 2
    assert 0 < p["fp64_fma_tflops"] < p["fp32_fma_tflops"]
