"""The measured FMA peaks are plausible for this GPU class: FP32 between a
quarter and 1.2 times the unit-count peak at the maximum clock (152 SMs x 128
lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s), FP64 well below FP32."""
import pytest

from paper_2508_03065_gb300 import api

pytestmark = pytest.mark.gpu


def test_measured_alu_peaks_are_plausible():
    import torch
    props = torch.cuda.get_device_properties(0)
    unit_peak = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    f32, f64 = api.measure_alu_peaks()
    assert 0.25 * unit_peak < f32 < 1.2 * unit_peak, (f32, unit_peak)
    assert 0.0 < f64 < 0.5 * f32, (f64, f32)
