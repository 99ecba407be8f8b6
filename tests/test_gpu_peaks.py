"""The FMA microbenchmark behind the roofline's denominators: plausible FP32 and FP64
throughput for a GB300 (152 SMs x 128 FP32 lanes at up to 2.07 GHz, 80.5 TFLOP/s, and an
FP64 rate a small fraction of it), measured twice within a few percent."""
import pytest

from gpu_common import nphc

pytestmark = pytest.mark.gpu


def test_fma_peaks_are_plausible_and_repeatable():
    nphc()
    from paper_1104_5497_gb300.peaks import alu_peak
    f32 = [alu_peak(32)["tflops"] for _ in range(2)]
    f64 = [alu_peak(64)["tflops"] for _ in range(2)]
    assert 30.0 < min(f32) and max(f32) < 90.0, f32
    assert 0.2 < min(f64) and max(f64) < 10.0, f64
    assert max(f32) / min(f32) < 1.1 and max(f64) / min(f64) < 1.1
    assert max(f64) < 0.2 * min(f32)
