"""qbvm_measure_peak: the measured FMA rates the ALU roofline is rated against.

The probe is a pure FMA-chain kernel; its rate must be positive, finite, of
the right order for this class of GPU (far below the nominal FP32 rate for
FP64 on GB300) and repeatable to a few percent.
"""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2107_06381_gb300 as Q  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    Q.build_library()
    return Q.load_library()


def test_fp64_and_fp32_fma_rates(lib):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clk = 2.2e9                                   # above any SM clock of this class of part
    f64 = Q.qbvm_measure_peak(Q.PEAK_FP64_FMA)
    f32 = Q.qbvm_measure_peak(Q.PEAK_FP32_FMA)
    assert 0 < f64 < f32
    # FP32: at most 128 FMA lanes per SM per clock; FP64 at most 64
    assert f32 <= sms * 128 * clk and f64 <= sms * 64 * clk
    # the probe must keep the pipes busy: at least a quarter of a 1-per-clock
    # FP64 rate and of a 64-lane FP32 rate at 1 GHz
    assert f64 >= 0.25 * sms * 1e9 and f32 >= 0.25 * sms * 64 * 1e9
    again = Q.qbvm_measure_peak(Q.PEAK_FP64_FMA)
    assert abs(again - f64) <= 0.1 * f64


def test_bad_kind_is_refused(lib):
    with pytest.raises(Q.QbvmError):
        Q.qbvm_measure_peak(7)
