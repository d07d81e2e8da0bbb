"""ade_alu_peaks: the measured FFMA and MUFU.RSQ issue rates that the interaction kernels' ALU
roof is checked against."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peak_probe_is_plausible(adelib):
    """FFMA at most 128 lanes per SM and RSQRT at most 32 per SM at up to 2.2 GHz, and at least
    half of 128 (FFMA) and 16 (RSQRT) lanes at 1 GHz."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ffma, rsq = adelib.alu_peaks()
    assert 0.5 * sms * 128 * 1.0e9 <= ffma <= sms * 128 * 2.2e9
    assert 0.5 * sms * 16 * 1.0e9 <= rsq <= sms * 32 * 2.2e9
