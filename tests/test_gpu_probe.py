"""The multiply-add rate probe that bench.py reports beside its ALU rooflines:
it runs through the C ABI and its rates are positive and below twice the
nominal unit rates (a kernel whose work the compiler dropped would read far
above them)."""
import pytest

import paper_2209_08437_gb300 as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NOMINAL_TFLOPS = {0: 2 * 152 * 2 * 2.07e-3, 1: 128 * 152 * 2 * 2.07e-3, 2: 128 * 152 * 2 * 2.07e-3}


@pytest.mark.parametrize("kind", [0, 1, 2], ids=["fp64", "fp32", "fp32-packed"])
def test_probe_rate_is_plausible(kind):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = 4 * sms
    buf = torch.zeros(blocks * 256, dtype=torch.float64 if kind == 0 else torch.float32, device="cuda")
    iters = 100 if kind == 0 else 2000
    S.sfac.sfac_probe_fma(kind, blocks, 2, buf)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    flops = S.sfac.sfac_probe_fma(kind, blocks, iters, buf)
    e1.record()
    torch.cuda.synchronize()
    tflops = flops / (e0.elapsed_time(e1) / 1e3) / 1e12
    print(f"kind {kind}: {tflops:.2f} TFLOP/s")
    assert 0 < tflops < 2 * NOMINAL_TFLOPS[kind] * 152 / sms
    assert bool(torch.isfinite(buf).all()) and float(buf.abs().max()) > 0


def test_probe_rejects_bad_arguments():
    buf = torch.zeros(256, device="cuda")
    for args in ((3, 1, 1), (0, 0, 1), (1, 1, 0)):
        with pytest.raises(S.SfacError):
            S.sfac.sfac_probe_fma(*args, buf)
