"""The ALU roofline's denominator, SMs x 128 lanes x SM clock, checked on the
device with an FP32 FMA loop: the loop cannot issue faster than that product at
the maximum clock, and a GB300 under the loop runs close to it."""
import pytest

from paper_2503_06757_gb300 import prrtc as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


def test_fma_loop_reaches_the_lane_clock_product():
    torch = pytest.importorskip("torch")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rate, ms = P.prrtc_alu_peak(16384)
    peak = sms * 128 * 2070e6  # maximum SM clock of a GB300
    print(f"FMA loop: {rate * 1e-12:.2f} T lane-ops/s over {ms:.3f} ms; {rate / peak:.3f} of {sms} x 128 x 2070 MHz")
    assert ms > 0.0
    assert rate <= 1.02 * peak
    assert rate >= 0.5 * peak


def test_bad_arguments_are_rejected():
    with pytest.raises(P.PrrtcError):
        P.prrtc_alu_peak(0)
