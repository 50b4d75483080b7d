"""The measured pipe peaks are plausible for a GB300: FP32 near the unit-count
figure (152 SMs x 128 lanes x 2 flop x clock), FP64 far below FP32."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_peaks():
    import paper_2309_13824_gb300 as g

    g.build()
    p = g.mesh_measure_pipe_peaks()
    nominal = p["sm_count"] * 128 * 2 * p["sm_clock_mhz"] * 1e6 / 1e12
    assert 0.5 * nominal < p["fp32_tflops"] < 1.1 * nominal, p
    assert 0 < p["fp64_tflops"] < 0.25 * p["fp32_tflops"], p
