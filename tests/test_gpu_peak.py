"""The measured FMA-pipe peaks (the Legendre kernels' roofline denominators):
plausible for a Blackwell part, consistent between the kernels, and the SM
count the device reports."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wfm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_08852_gb300 import build
    build.build()
    from paper_1702_08852_gb300 import wf
    return wf, torch


def test_alu_peaks_are_plausible(wfm):
    wf, torch = wfm
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f64, _, n0 = wf.wf_alu_peak(0, 2)
    f32, _, n1 = wf.wf_alu_peak(1, 2)
    f32x2, _, n2 = wf.wf_alu_peak(2, 2)
    assert n0 == n1 == n2 == sms
    # at most 128 FP32 lanes x 2 flops x 2.2 GHz per SM; FP64 far below FP32
    ceiling = sms * 128 * 2 * 2.2e9 / 1e12
    assert 0.3 * ceiling < max(f32, f32x2) <= 1.05 * ceiling
    assert 0.0 < f64 < 0.5 * f32


def test_alu_peak_rejects_bad_arguments(wfm):
    wf, _ = wfm
    with pytest.raises(wf.WFError) as e:
        wf.wf_alu_peak(3, 1)
    assert e.value.status == wf.WF_ERR_ARG
