"""The multiply-add rate probe that bench.py reports beside its ALU rooflines:
it runs through the C ABI and its rates are positive and below twice the
nominal unit rates (a kernel whose work the compiler dropped would read far
above them)."""
import numpy as np
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


def _jq_values(dtype):
    """FP64: [-1.5, 1.5], wide normal samples and special values up to 1e18.
    FP32: [-1.5, 1.5] only (the increment form's range: beyond it the flow
    shrinks v by a large factor and the increment cancels most of v)."""
    rng = np.random.default_rng(7)
    if dtype == np.float64:
        v = np.concatenate([np.linspace(-1.5, 1.5, 200001), rng.normal(0.0, 3.0, 50000),
                            [0.0, -0.0, 1.0, -1.0, 1e-300, -1e-300, 5e-324, -5e-324, 1e10, -1e10, 1e18, -1e18]])
    else:
        v = np.concatenate([np.linspace(-1.5, 1.5, 200001), np.clip(rng.normal(0.0, 0.6, 50000), -1.5, 1.5),
                            [0.0, -0.0, 1.0, -1.0, 1e-30, -1e-30]])
    return v.astype(dtype)


def _ulp_errors(out, v, E, om):
    """|out - J^Q(v)| in units in the last place of J^Q(v), the flow evaluated
    in extended precision from the same v, E and 1 - E the kernel sees."""
    ld = np.longdouble
    ref = v.astype(ld) / np.sqrt(ld(E) + ld(om) * v.astype(ld) ** 2)
    ref_r = ref.astype(out.dtype)
    ulp = np.spacing(np.abs(ref_r)).astype(ld)
    return np.abs(out.astype(ld) - ref) / ulp


@pytest.mark.parametrize("s2", [1e-3, 2e-3, 4e-3, 0.1, 2.0, 80.0])
def test_fp64_flow_within_three_ulp(s2):
    """J^Q_s(v) = v / sqrt(E + (1 - E) v^2), E = e^{-2s} (the exact solution of
    u' = u - u^3, Sec. 2.2) as the FP64 passes evaluate it: within 3 units in
    the last place of the extended-precision value over v in [-1.5, 1.5],
    wide normal samples and the special values."""
    E, om = float(np.exp(-s2)), float(-np.expm1(-s2))
    v = _jq_values(np.float64)
    vd = torch.tensor(v, device="cuda")
    out = torch.empty_like(vd)
    S.sfac.sfac_probe_jq(S.SFAC_FP64, vd, out, E, om)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    err = _ulp_errors(o, v, E, om)
    print(f"2s={s2}: max {float(err.max()):.2f} ulp, mean {float(err.mean()):.3f}")
    assert float(err.max()) <= 3.0
    assert np.all(o[v == 0.0] == 0.0)
    assert np.array_equal(np.sign(o), np.sign(v))


@pytest.mark.parametrize("s2,bound", [(1e-3, 1.0), (2e-3, 1.0), (1e-2, 1.0), (0.5, 6.0)])
def test_fp32_flow_increment_form(s2, bound):
    """The FP32 passes' J^Q (v plus its increment, from 1 - E alone) on
    [-1.5, 1.5]: within one unit in the last place for the small steps of the
    workloads (the increment is about s |v|, so its few-ulp approximations
    vanish in the final rounding), within a few for 2s = 0.5."""
    om32 = np.float32(-np.expm1(-s2))
    om = float(om32)
    v = _jq_values(np.float32)
    vd = torch.tensor(v, device="cuda")
    out = torch.empty_like(vd)
    S.sfac.sfac_probe_jq(S.SFAC_FP32, vd, out, 1.0 - om, om)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    err = _ulp_errors(o, v, 1.0 - om, om)
    print(f"2s={s2}: max {float(err.max()):.2f} ulp, mean {float(err.mean()):.3f}")
    assert float(err.max()) <= bound


def test_flow_probe_odd_count_and_in_place():
    """An odd number of values (the last thread holds one) and out == v."""
    v = torch.linspace(-1.2, 1.2, 1001, dtype=torch.float64, device="cuda")
    ref = v.clone()
    S.sfac.sfac_probe_jq(S.SFAC_FP64, ref, ref, float(np.exp(-2e-3)), float(-np.expm1(-2e-3)))
    out = torch.empty_like(v)
    S.sfac.sfac_probe_jq(S.SFAC_FP64, v, out, float(np.exp(-2e-3)), float(-np.expm1(-2e-3)))
    torch.cuda.synchronize()
    assert torch.equal(ref, out)
    assert float(out[-1]) != 0.0
