"""The integer-pipe rate measurement behind the sweep kernels' roofline."""
import pytest

pytestmark = pytest.mark.gpu


def test_integer_peaks_are_plausible():
    import torch
    from paper_2311_09275_gb300 import isg
    props = torch.cuda.get_device_properties(0)
    r = isg.isg_integer_peaks()
    # per SM and cycle at most 128 lanes can retire an instruction (4 schedulers x 32),
    # and no pipe here is slower than 4 lanes per scheduler
    clk = 2.2e9
    for key in ("lop3_per_s", "mad_wide_per_s"):
        per_sm_cycle = r[key] / props.multi_processor_count / clk
        assert 16 <= per_sm_cycle <= 128 * 1.05, (key, r[key])


def test_philox_rates_are_plausible():
    from paper_2311_09275_gb300 import isg
    r = isg.isg_philox_rates()
    # 4 widening multiplies per uniform on a quarter-rate pipe: at most ~1.3e13/s on 152 SMs
    assert 1e11 < r["masked_per_s"] <= r["uniforms_per_s"] * 1.05 < 2e13, r
