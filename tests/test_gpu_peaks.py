"""The arithmetic-rate microbenchmark behind the rooflines (mh_measure_peaks):
the measured rates lie within reach of the unit-count peaks of a GB300
(FP64: 2 lanes x 2 flops per SM per clock; FP32: 128 lanes x 2) at clocks up
to 2.07 GHz, and no kernel beats its unit count."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_measured_alu_peaks(mh_pkg=None):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_02501_gb300 as mh
    mh.build_library()
    p = mh.measure_peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    fp64_max = n_sm * 2 * 2 * 2.2e9 / 1e12           # 2.2 GHz: above any clock of the part
    fp32_max = n_sm * 128 * 2 * 2.2e9 / 1e12
    assert 0.3 * fp64_max < p["fp64_tflops"] <= fp64_max, p
    assert 0.3 * fp32_max < p["fp32_tflops"] <= fp32_max, p
    assert 0.3 * fp32_max < p["fp32x2_tflops"] <= fp32_max, p
    assert p["rsqrt_tera_per_s"] > 0, p
