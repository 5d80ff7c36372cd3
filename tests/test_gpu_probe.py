"""The issue-rate probe behind the path kernels' roofline: on the GPU at hand
the FP32 fused multiply-add rate must come close to (and not exceed) one warp
instruction per scheduler per cycle at the maximum SM clock, and the SFU rate
must sit well below it (the SFU pipe is narrower)."""
import pytest

pytestmark = pytest.mark.gpu


def test_issue_rates():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    torch.cuda.init()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 4 * 32 * 2.07e9  # thread-instructions per second at the maximum SM clock
    fma, ms = pdd.pdd_debug_issue_rate(0, 4096)
    assert ms > 0
    assert 0.5 * peak < fma < 1.05 * peak, (fma, peak)
    sfu, _ = pdd.pdd_debug_issue_rate(2, 1024)
    assert 0.0 < sfu < 0.5 * fma
    with pytest.raises(pdd.PddError):
        pdd.pdd_debug_issue_rate(7, 10)
