"""rbe_probe_peaks: the measured unit rates behind the bench's rooflines are
plausible for this part (special-function unit 16 sin/cos results per SM per
clock and 128 FP32 FMA lanes per SM nominally; a probe that is issue- or
dependency-bound reads lower, one that reads far higher is not measuring)."""
import pytest

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_probe_peaks_plausible():
    need_gpu()
    import __graft_entry__
    __graft_entry__.build()
    import paper_2010_01559_gb300 as rbe
    pk = rbe.probe_peaks()
    print(pk)
    assert pk["sms"] >= 1
    assert 4.0 <= pk["sfu_per_clk_sm"] <= 17.0
    assert 32.0 <= pk["ffma_per_clk_sm"] <= 130.0
    assert 300.0 <= pk["sm_clock_mhz"] <= 3000.0
