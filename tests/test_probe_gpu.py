"""Issue-rate probes behind the C ABI (measurement infrastructure for the
walk's roofline): each kind runs, counts its operations, and measures a
throughput inside what one SM can issue."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_27604_b300 import api as a
    return a


def test_probes_run_and_measure_plausible_rates(api):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = sms * 8
    sink = torch.zeros(blocks * 256, dtype=torch.float32, device="cuda")
    rates = {}
    for kind in api.PROBE_KINDS:
        iters = 1 << (12 if kind in ("mufu_lg2", "philox") else 15)
        api.probe(kind, 16, blocks, sink)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ops = api.probe(kind, iters, blocks, sink)
        b.record()
        torch.cuda.synchronize()
        per = {"ffma2": 16, "philox": 4}.get(kind, 8)
        assert ops == blocks * 256 * iters * per
        rates[kind] = ops / (a.elapsed_time(b) / 1e3) / sms / 2.1e9  # lanes/clk/SM, clock <= 2.1 GHz
        if kind in ("ffma", "ffma2", "mufu_lg2"):
            assert torch.isfinite(sink).all(), kind
    print({k: round(v, 1) for k, v in rates.items()})
    # an SM has 4 schedulers issuing at most one 32-lane instruction per clock
    assert rates["ffma"] <= 4 * 32 * 1.05 and rates["ffma"] > 32
    assert rates["mufu_lg2"] < rates["ffma"]
    # a Philox4x32-10 block holds 20 32x32-bit products and 20 three-input
    # XORs, so whole blocks issue far slower than single multiply-adds
    assert 0 < rates["philox"] < rates["imad"] / 10
    with pytest.raises(api.SSSError):
        api.probe("ffma", 0, blocks, sink)
