"""The arithmetic-throughput entry point (measurement support for the roofline of the kernels
bound by arithmetic rather than memory)."""
import pytest

from paper_2608_23786_gb300 import mclbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mclbm.load(build_if_missing=True)


def test_alu_rate_measures_the_pipes():
    """mclbm_alu_rate (the arithmetic ceilings behind the FP64-bound kernels' roofline): every kind
    returns a positive rate with a timed launch; FP32 fma outruns FP64 fma on this class of GPU,
    and the reciprocal unit is slower than the FP32 fma pipe.  Invalid kinds are rejected."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    rates = {}
    for kind in mclbm.ALU_KINDS:
        r, ms = mclbm.mclbm_alu_rate(kind, 16, sink.data_ptr())
        assert r > 0 and ms > 0, kind
        rates[kind] = r
    assert rates["fp32_fma"] > 4 * rates["fp64_fma"]
    assert rates["fp32_rcp"] < rates["fp32_fma"]
    assert float(sink.cpu()[0]) == 0.0  # the chains never reach the sink's trigger value
    with pytest.raises(mclbm.MclbmError) as e:
        mclbm.mclbm_alu_rate(7, 16, sink.data_ptr())
    assert e.value.status == "INVALID_ARG"
