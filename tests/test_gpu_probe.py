"""GPU: the FMA throughput probe behind the arithmetic roofline's denominator (gbr_alu_peak).

B300 nominal figures: FP64 about 1.2-1.25 TFLOP/s (2 FP64 FMA lanes per SM-clock x 148 SMs at
up to 2.032 GHz), FP32 about 77 TFLOP/s (128 lanes per SM-clock).  The probe must land near
them (a broken probe reads far off) and FP32 must be far faster than FP64 on this part."""
import pytest

from paper_2303_10785_b300 import gbr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def test_alu_peak_probe_reads_near_the_nominal_rates():
    f64, ms64 = gbr.alu_peak("fp64")
    f32, ms32 = gbr.alu_peak("mixed")
    assert ms64 > 1.0 and ms32 > 1.0
    assert 0.6 < f64 < 1.6, f64
    assert 30.0 < f32 < 100.0, f32
    assert f32 > 20 * f64
    assert gbr.lib().gbr_alu_peak(7, None, None, None) == gbr.GBR_EINVAL
