"""The FP32 FMA probe (sw_measure_fp32_fma): the measured denominator of the
ALU-bound rooflines lies between a third of and just above the unit-count
peak (SMs x 128 FP32 lanes x 2 flops x the maximum SM clock)."""
import pytest

from paper_2503_13756_gb300 import swalign

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fp32_fma_probe_is_near_the_unit_count_peak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tf, ms = swalign.measure_fp32_fma(0)
    props = torch.cuda.get_device_properties(0)
    mhz = getattr(props, "clock_rate", 0) / 1e3 or 2070.0
    nominal = props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12
    assert ms > 0
    assert 0.33 * nominal < tf < 1.1 * nominal, (tf, nominal)
