"""sfac_step_host on host memory (the end-to-end entry point).

Pinned host buffers are mapped into the device's address space. Where the
first and the last pass have 4096 line pairs or more, the first pass of a call
reads the field from the mapped buffer and the last pass writes the result
back into it (SFAC_HOST_MAPPED), or, for an FP32 last axis longer than 512
points, a copy brings the result back (SFAC_HOST_MAPPED_IN); other fields,
pageable buffers and the whole-call launch of small grids are copied in and
out (SFAC_HOST_COPY). Every route runs the same arithmetic on the same lines
as sfac_step on a device field, so the results must be the same bits, for
every kernel route: FP64 CTA passes, FP32 warp, 1024-point CTA and
2048-point persistent passes,
zero-padded passes, and an FP32 last axis that the device route runs staged
(TMA) and the mapped route on 256-thread CTAs (rows of 64 bytes or more)."""
import numpy as np
import pytest

import paper_2209_08437_gb300 as S
import sfac_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COPY, MAPPED, MAPPED_IN = S.SFAC_HOST_COPY, S.SFAC_HOST_MAPPED, S.SFAC_HOST_MAPPED_IN

CASES = [
    ((32, 256, 32), S.SFAC_FP64, MAPPED),
    ((40, 256, 48), S.SFAC_FP64, MAPPED),       # zero-padded first and last axis
    ((64, 128, 256), S.SFAC_FP32, MAPPED),      # last axis staged on the device route
    ((48, 256, 80), S.SFAC_FP32, MAPPED),       # zero-padded first and last axis
    ((1024, 64, 128), S.SFAC_FP32, MAPPED),     # 1024-point CTA pass first
    ((32, 256, 1024), S.SFAC_FP32, MAPPED_IN),  # 1024-point last axis: result copied back
    ((2048, 16, 512), S.SFAC_FP32, MAPPED),     # 2048-point persistent CTAs read the host buffer
    ((256, 64), S.SFAC_FP64, COPY),             # 32 line pairs in the last pass
    ((64, 64), S.SFAC_FP32, COPY),              # small grid (whole-call launch from 2 steps)
    ((512,), S.SFAC_FP32, COPY),                # one line
]


def _run(n, prec, nsteps, route):
    dim = len(n)
    prob = I.Problem(n=n, alpha=(1.3, 1.7, 1.5)[:dim], eps=0.07, tau=2e-3)
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    u0 = I.random_field(prob, 11 + dim, -0.95, 0.95)
    with S.Plan.for_problem(prob, prec) as plan:
        u = torch.tensor(np.ascontiguousarray(u0), dtype=dt, device="cuda")
        plan.step(u, nsteps)
        plan.check()
        want = u.cpu().numpy()
        pinned = torch.tensor(np.ascontiguousarray(u0), dtype=dt).pin_memory()
        assert plan.host_route(pinned.numpy(), nsteps) == route
        plan.step_host(pinned.numpy(), nsteps)
        pageable = np.array(u0, dtype=want.dtype, copy=True)
        assert plan.host_route(pageable, nsteps) == COPY
        plan.step_host(pageable, nsteps)
        assert np.array_equal(pinned.numpy(), want)
        assert np.array_equal(pageable, want)
        # again on the same pinned buffer: the call reads what the last one wrote
        plan.step_host(pinned.numpy(), 1)
        plan.step(u, 1)
        plan.check()
        assert np.array_equal(pinned.numpy(), u.cpu().numpy())


@pytest.mark.parametrize("n,prec,route", CASES, ids=str)
def test_host_routes_match_the_device_call(n, prec, route):
    _run(n, prec, 3, route)


@pytest.mark.parametrize("n,prec,route", [CASES[0], CASES[2], CASES[5]], ids=str)
def test_host_routes_one_step(n, prec, route):
    _run(n, prec, 1, route)


def test_zero_steps_and_small_grids_take_the_copies():
    prob = I.Problem(n=(64, 32), alpha=(1.4, 1.6), eps=0.1, tau=1e-3)
    u0 = I.random_field(prob, 3)
    with S.Plan.for_problem(prob, S.SFAC_FP64) as plan:
        pinned = torch.tensor(u0).pin_memory()
        assert plan.host_route(pinned.numpy(), 0) == COPY
        plan.step_host(pinned.numpy(), 0)
        assert np.array_equal(pinned.numpy(), u0)
    big = I.Problem(n=(32, 256, 32), alpha=(1.4, 1.6, 1.5), eps=0.1, tau=1e-3)
    with S.Plan.for_problem(big, S.SFAC_FP64) as plan:
        pinned = torch.zeros(big.shape, dtype=torch.float64).pin_memory()
        assert plan.host_route(pinned.numpy(), 0) == COPY
        assert plan.host_route(pinned.numpy(), 1) == MAPPED
        view = pinned.numpy().reshape(-1)[1:]          # not 16-byte aligned
        assert plan.host_route(view, 1) == COPY
