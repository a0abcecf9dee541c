"""The FP32 strided pass with TMA-staged tiles (SFAC_KERNEL_STAGED).

Strided passes of FP32 plans with line lengths 32..512 copy whole tiles of the
field (32 columns, or 16 from length 256, by all rows of a slab) into shared
memory with TMA and run the fused pass of Sec. 2.2 on them, when the pass has at
least as many tiles as the GPU has SMs. These tests check which passes take that
route, that a staged pass computes exactly what the warp kernel computes on the
same lines, and the FP32 parity bar (max-norm error <= 1e-5 against the FP64
oracle) on shapes with several tiles, ragged last tiles (a stride that is not a
multiple of the tile width) and both tile widths.
"""
import numpy as np
import pytest

import paper_2209_08437_gb300 as S
import sfac_inputs as I
from oracle import sfac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CTA, WARP, STAGED = S.SFAC_KERNEL_CTA, S.SFAC_KERNEL_WARP, S.SFAC_KERNEL_STAGED


def dev(u, prec=S.SFAC_FP32):
    dt = torch.float32 if prec == S.SFAC_FP32 else torch.float64
    return torch.tensor(np.ascontiguousarray(u), dtype=dt, device="cuda")


@pytest.mark.parametrize("n,prec,expect", [
    ((256, 256, 256), S.SFAC_FP32, [WARP, STAGED, STAGED]),
    ((256, 256, 256), S.SFAC_FP64, [CTA, CTA, CTA]),
    ((1024, 1024), S.SFAC_FP32, [CTA, CTA]),
    ((48, 256, 64), S.SFAC_FP32, [WARP, STAGED, STAGED]),  # axis 2 stride 48: ragged last tiles
    ((8, 256, 256), S.SFAC_FP32, [CTA, WARP, WARP]),       # stride 8 < tile width 16; 128 tiles
    ((48, 256), S.SFAC_FP32, [WARP, WARP]),                # 3 tiles: fewer than the SMs
    ((64, 512), S.SFAC_FP32, [WARP, WARP]),                # 4 tiles
    ((32, 64, 160), S.SFAC_FP32, [WARP, STAGED, WARP]),    # n = 160: zero-padded pass, L = 512
    ((63, 64), S.SFAC_FP32, [WARP, WARP]),                 # odd stride: zero-padded pass
], ids=str)
def test_kernel_routing(n, prec, expect):
    prob = I.Problem(n=n, alpha=(1.5,) * len(n), eps=0.1, tau=0.01)
    with S.Plan.for_problem(prob, prec) as plan:
        u = torch.zeros(plan.shape, dtype=torch.float32 if prec == S.SFAC_FP32 else torch.float64,
                        device="cuda")
        assert [plan.kernel(ax, u) for ax in range(len(n))] == expect
        # a field that is not 16-byte aligned cannot be staged
        flat = torch.zeros(u.numel() + 4, dtype=u.dtype, device="cuda")
        assert all(plan.kernel(ax, flat[1:]) != STAGED for ax in range(len(n)))


@pytest.mark.parametrize("n", [(32, 256, 80), (64, 128, 80), (32, 32, 160), (64, 64, 80), (16, 512, 160)], ids=str)
def test_staged_pass_equals_warp_pass_on_the_same_lines(n):
    """Axis 2 of the field (staged) and axis 1 of its transpose (warp kernel,
    contiguous lines) form the same complex lines from the same column/row
    pairs and run the same arithmetic; results agree to FP32 rounding."""
    n0, n1, n2 = n
    alpha = (1.35, 1.65, 1.5)
    prob = I.Problem(n=n, alpha=alpha, eps=0.07, tau=0.01)
    u0 = I.random_field(prob, 77, -1.0, 1.0).astype(np.float32)        # shape (n2, n1, n0)
    probT = I.Problem(n=(n1, n0, n2), alpha=(alpha[1], alpha[0], alpha[2]), eps=0.07, tau=0.01)
    with S.Plan.for_problem(prob, S.SFAC_FP32) as p, S.Plan.for_problem(probT, S.SFAC_FP32) as pT:
        u = dev(u0)
        uT = dev(np.transpose(u0, (0, 2, 1)))                                # shape (n2, n0, n1)
        assert p.kernel(1, u) == STAGED and pT.kernel(0, uT) == WARP
        for jin, jout in [(0, 0), (1, 2)]:
            p.axis_pass(u, 1, jin, jout)
            pT.axis_pass(uT, 0, jin, jout)
        p.check()
        a = u.double().cpu().numpy()
        b = np.transpose(uT.double().cpu().numpy(), (0, 2, 1))
    diff = float(np.abs(a - b).max())
    print(f"{n}: staged vs warp kernel max diff {diff:.3e} (bitwise: {diff == 0.0})")
    assert diff <= 2e-7 * max(1.0, float(np.abs(b).max()))


@pytest.mark.parametrize("n", [(32, 32, 192), (48, 64, 80), (32, 128, 160), (16, 256, 160), (40, 256, 64),
                               (64, 512, 40)], ids=str)
def test_staged_steps_match_oracle(n):
    """FP32 steps with staged strided passes against the FP64 oracle: max-norm
    error <= 1e-5."""
    prob = I.Problem(n=n, alpha=(1.25, 1.75, 1.45)[: len(n)], eps=0.06, tau=2e-3)
    u0 = I.random_field(prob, 31, -0.95, 0.95)
    u32 = u0.astype(np.float32)
    ref = O.solve(prob, u32.astype(np.float64), 4)
    with S.Plan.for_problem(prob, S.SFAC_FP32) as plan:
        u = dev(u32)
        assert any(plan.kernel(ax, u) == STAGED for ax in range(len(n)))
        plan.step(u, 4)
        plan.check()
        got = u.double().cpu().numpy()
    err = float(np.abs(got - ref).max())
    print(f"{n}: FP32 staged max-norm error {err:.3e}")
    assert err <= 1e-5


def test_step_host_checks_status():
    prob = I.Problem(n=(32, 256, 80), alpha=(1.5, 1.5, 1.5), eps=0.1, tau=1e-3)
    u0 = I.random_field(prob, 5, -0.9, 0.9).astype(np.float32)
    with S.Plan.for_problem(prob, S.SFAC_FP32) as plan:
        h = np.array(u0, copy=True)
        plan.step_host(h, 3)                      # runs sfac_plan_check internally
        u = dev(u0)
        plan.step(u, 3)
        plan.check()
        assert np.array_equal(h, u.cpu().numpy())


def test_bounded_tile_wait_runs_out_and_the_plan_stays_usable():
    """Test hook: the first tile wait of every CTA goes to a barrier that nothing
    completes. Each CTA gives up after the wait limit (1e5 cycles here), records
    the timeout, waits for its copies in flight and returns; sfac_plan_check
    reports SFAC_ETIMEOUT once and clears it, and the plan then runs normally
    (same result as a fresh plan)."""
    prob = I.Problem(n=(32, 256, 80), alpha=(1.4, 1.6, 1.5), eps=0.08, tau=1e-3)
    u0 = I.random_field(prob, 9, -0.9, 0.9).astype(np.float32)
    with S.Plan.for_problem(prob, S.SFAC_FP32) as plan, S.Plan.for_problem(prob, S.SFAC_FP32) as fresh:
        u = dev(u0)
        assert plan.kernel(1, u) == STAGED
        S.sfac_plan_set_wait_limit(plan.handle, 100_000, 1)
        plan.axis_pass(u, 1)
        with pytest.raises(S.SfacError) as ei:
            plan.check()
        assert ei.value.status == S.sfac.SFAC_ETIMEOUT
        plan.check()                                  # the flag was cleared
        S.sfac_plan_set_wait_limit(plan.handle, 1 << 32, 0)
        a, b = dev(u0), dev(u0)
        plan.step(a, 2)
        fresh.step(b, 2)
        plan.check()
        assert torch.equal(a, b)
