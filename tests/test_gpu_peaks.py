"""The integer-pipe rate measurement behind the sweep kernels' roofline."""
import pytest

pytestmark = pytest.mark.gpu


def test_integer_peaks_are_plausible():
    import torch
    from paper_2311_09275_gb300 import isg
    props = torch.cuda.get_device_properties(0)
    r = isg.isg_integer_peaks()
    # per SM and cycle: the logic pipe retires at most 64 lanes (4 schedulers x 16),
    # the widening multiply at most 32 (4 schedulers x 8); neither is slower than 4
    # lanes per scheduler (clk: above the 2.07 GHz maximum, so a lower bound per cycle)
    clk = 2.2e9
    for key, top in (("lop3_per_s", 64), ("mul_wide_per_s", 32)):
        per_sm_cycle = r[key] / props.multi_processor_count / clk
        assert 16 <= per_sm_cycle <= top * 1.1, (key, r[key])


def test_philox_rates_are_plausible():
    from paper_2311_09275_gb300 import isg
    r = isg.isg_philox_rates()
    # 4 widening multiplies per uniform on a quarter-rate pipe: at most ~1.3e13/s on 152 SMs
    assert 1e11 < r["masked_per_s"] <= r["uniforms_per_s"] * 1.05 < 2e13, r
