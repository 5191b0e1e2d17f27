"""The peak probes that give the event kernels' roofline its denominators
(qed_peak_probe): each runs, and the rates are those of a GB300-class part
(152 SMs near 2 GHz).  GPU only."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2008_10468_gb300 import qed  # noqa: E402


def test_peak_probes():
    rates = {k: qed.peak_probe(k, 1 << 14)[0] for k in
             (qed.PROBE_MUL32, qed.PROBE_FMA32, qed.PROBE_EX2, qed.PROBE_ALU)}
    print("peak probes (ops/s):", rates)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clk = 2.1e9
    # per SM and clock: FMA at most 128 lanes x 2 flops, multiplies at most 128
    # lanes x 2 words, exp2 at most 32 lanes, the ALU at most 128 lanes x 2
    assert 0.2 * sms * clk * 64 * 2 < rates[qed.PROBE_FMA32] <= sms * clk * 128 * 2
    assert 0.1 * sms * clk * 32 * 2 < rates[qed.PROBE_MUL32] <= sms * clk * 128 * 2
    assert 0.1 * sms * clk * 8 < rates[qed.PROBE_EX2] <= sms * clk * 32
    assert 0.1 * sms * clk * 64 * 2 < rates[qed.PROBE_ALU] <= sms * clk * 128 * 2
    with pytest.raises(qed.QEDError):
        qed.peak_probe(7)
