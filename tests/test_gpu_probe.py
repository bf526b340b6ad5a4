"""GPU: the FMA throughput probe behind the arithmetic roofline's denominator (gbr_alu_peak), and
the FP64 reciprocal the kernels use in place of divisions, against the division (gbr_check_rcp).

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


def test_fp64_reciprocal_is_within_one_ulp_of_the_division():
    # Newton's method from the approximate reciprocal: within one unit in the last place of the
    # correctly rounded 1/x over 2^27 random normal x (and 1/x normal), for two seeds
    for seed in (0, 12345):
        assert gbr.check_rcp(1 << 27, seed) <= 1
    assert gbr.lib().gbr_check_rcp(0, 0, None, None) == gbr.GBR_EINVAL
