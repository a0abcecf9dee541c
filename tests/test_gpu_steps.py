"""GPU tests of the whole-call launch for small grids (csrc/sfac_steps.cu):
a call of two or more steps on a grid of at most 65536 unknowns whose axes are
spectral passes of 32..256 points runs in one cooperative launch with a
grid-wide barrier between passes. Checked against the CPU FP64 oracle, against
the per-step launches, and for its bounded barrier wait."""
import numpy as np
import pytest

import paper_2209_08437_gb300 as S
import sfac_inputs as I
from oracle import sfac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = [(64, 64), (32, 128), (256, 64), (128, 256), (32, 32, 32), (64, 32, 32), (256,)]


def dev(u, prec):
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    return torch.tensor(np.ascontiguousarray(u), dtype=dt, device="cuda")


def test_which_calls_take_the_whole_call_launch():
    cases = [((64, 64), 2, S.SFAC_STEP_WHOLE), ((64, 64), 1, S.SFAC_STEP_PASSES),
             ((32, 32, 32), 10, S.SFAC_STEP_WHOLE), ((1024, 64), 5, S.SFAC_STEP_PASSES),
             ((16, 64), 5, S.SFAC_STEP_PASSES), ((63, 64), 5, S.SFAC_STEP_PASSES),
             ((256, 512), 5, S.SFAC_STEP_PASSES)]
    for n, k, want in cases:
        prob = I.Problem(n=n, alpha=(1.4, 1.6, 1.5)[: len(n)], eps=0.1, tau=1e-2)
        for prec in (S.SFAC_FP64, S.SFAC_FP32):
            with S.Plan.for_problem(prob, prec) as plan:
                assert plan.step_kernel(k) == want, (n, k, prec)


@pytest.mark.parametrize("n", SMALL, ids=str)
@pytest.mark.parametrize("prec", [S.SFAC_FP64, S.SFAC_FP32], ids=["fp64", "fp32"])
def test_whole_call_matches_oracle(n, prec):
    prob = I.Problem(n=n, alpha=(1.3, 1.7, 1.5)[: len(n)], eps=0.08, tau=0.01)
    u0 = I.random_field(prob, 31, -0.9, 0.9)
    k = 6
    ref = O.Scheme.for_problem(prob).run(u0, k)
    src = u0 if prec == S.SFAC_FP64 else np.asarray(u0, np.float32).astype(np.float64)
    with S.Plan.for_problem(prob, prec) as plan:
        assert plan.step_kernel(k) == S.SFAC_STEP_WHOLE
        u = dev(src, prec)
        plan.step(u, k)
        plan.check()
        got = u.double().cpu().numpy()
    if prec == S.SFAC_FP64:
        assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-12
    else:
        assert np.abs(got - ref).max() <= 1e-5


@pytest.mark.parametrize("n", [(64, 64), (32, 32, 32)], ids=str)
def test_whole_call_equals_per_step_calls(n):
    """k steps in one call (one launch, J^Q halves merged between steps) and k
    calls of one step (per-pass launches, no merging) are the same scheme."""
    prob = I.Problem(n=n, alpha=(1.2, 1.8, 1.5)[: len(n)], eps=0.1, tau=0.02)
    u0 = I.random_field(prob, 32)
    with S.Plan.for_problem(prob) as plan:
        a, b = dev(u0, S.SFAC_FP64), dev(u0, S.SFAC_FP64)
        plan.step(a, 9)
        for _ in range(9):
            plan.step(b, 1)
        plan.check()
    assert float((a - b).abs().max() / b.abs().max()) <= 1e-14


def test_barrier_wait_runs_out_and_the_plan_stays_usable():
    """Test hook: the first barrier wait of every CTA waits for a generation
    that never comes. Each CTA gives up after the wait limit, records the
    timeout and returns; sfac_plan_check reports SFAC_ETIMEOUT once, and the
    plan then runs normally (same result as a fresh plan)."""
    prob = I.Problem(n=(64, 64), alpha=(1.4, 1.6), eps=0.1, tau=1e-2)
    u0 = I.random_field(prob, 33)
    with S.Plan.for_problem(prob) as plan, S.Plan.for_problem(prob) as fresh:
        u = dev(u0, S.SFAC_FP64)
        S.sfac_plan_set_wait_limit(plan.handle, 100_000, 1)
        plan.step(u, 4)
        with pytest.raises(S.SfacError) as ei:
            plan.check()
        assert ei.value.status == S.sfac.SFAC_ETIMEOUT
        plan.check()                                  # the flag was cleared
        S.sfac_plan_set_wait_limit(plan.handle, 1 << 32, 0)
        a, b = dev(u0, S.SFAC_FP64), dev(u0, S.SFAC_FP64)
        plan.step(a, 4)
        fresh.step(b, 4)
        plan.check()
        assert torch.equal(a, b)


def test_whole_call_in_a_cuda_graph():
    """The cooperative launch can be captured and replayed; each replay runs
    the call again."""
    prob = I.Problem(n=(64, 64), alpha=(1.5, 1.5), eps=0.1, tau=0.01)
    u0 = I.random_field(prob, 34)
    with S.Plan.for_problem(prob) as plan:
        u = dev(u0, S.SFAC_FP64)
        ref = dev(u0, S.SFAC_FP64)
        plan.step(ref, 5)
        plan.step(ref, 5)
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                plan.step(u, 5, stream=side.cuda_stream)
        torch.cuda.synchronize()
        u.copy_(dev(u0, S.SFAC_FP64))
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        plan.check()
    assert torch.equal(u, ref)
