"""The measured ALU peaks that the ALU-bound composites are reported against
(the micro-kernels of gs3_measure_alu_peak)."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peak_is_measured_and_plausible(gs3):
    import torch
    from paper_2410_11419_gb300 import _native as N
    ffma, ex2 = N.gs3_measure_alu_peak(3)
    props = torch.cuda.get_device_properties(0)
    # an SM issues at most 128 FP32 FMAs (256 FLOP) per clock; clocks stay below 3 GHz
    ceiling = props.multi_processor_count * 256 * 3.0e9 / 1e12
    assert 0.25 * ceiling < ffma < ceiling
    # ex2 runs on the special-function units, a fraction of the FMA rate
    assert 0.0 < ex2 * 1e9 < 0.5 * ffma * 1e12
