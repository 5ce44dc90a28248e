"""The measured ALU peaks (rx_measure_alu_peak) that the SIMT-bound stages'
rooflines divide by: FP32 near 152 SMs x 128 lanes x 2 flop x the SM clock,
FP64 far below it, and the FMA count independent of the chain length."""
import pytest

from chain_helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_measured_fp32_and_fp64_fma_peaks():
    from paper_2104_06311_gb300.rx import RxError, measure_alu_peak
    nominal = 152 * 128 * 2 * 2.07e9 / 1e12          # 80.5 TFLOP/s at the maximum clock
    f32 = max(measure_alu_peak("fp32", 32768)[0] for _ in range(3))
    f32_short = max(measure_alu_peak("fp32", 8192)[0] for _ in range(3))
    f64 = max(measure_alu_peak("fp64", 512)[0] for _ in range(2))
    print(f"FP32 {f32:.1f} TFLOP/s ({f32 / nominal:.3f} of nominal at 2070 MHz), FP64 {f64:.3f} TFLOP/s")
    assert 0.5 * nominal < f32 < 1.05 * nominal
    assert abs(f32_short / f32 - 1) < 0.15              # a rate, not a launch overhead
    assert 0.05 < f64 < f32 / 4
    with pytest.raises(RxError):
        measure_alu_peak("fp32", 7)                     # not a multiple of 8
