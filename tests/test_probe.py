"""The measured FMA rates (pastila_probe_fma) that the bench reports beside the
derived FP32 peak: FP32 near 148 SMs x 128 lanes x 2 FLOP x the SM clock, and
FP64 far below it on this GPU."""
import pytest

pytestmark = pytest.mark.gpu

DERIVED_FP32_TFLOPS = 148 * 128 * 2 * 2032e6 / 1e12


def test_probe_fma_rates(lib):
    from paper_2401_13680_b300 import pastila
    f32, f64 = pastila.probe_fma(0)
    assert 0.4 * DERIVED_FP32_TFLOPS < f32 < 1.05 * DERIVED_FP32_TFLOPS
    assert 0 < f64 < f32 / 8
    with pytest.raises(pastila.PastilaError, match="EINVAL"):
        pastila.probe_fma(999)
