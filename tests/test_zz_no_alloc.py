"""The allocation-free batched launch, sfac_batch_launch_noalloc.

Some callers may not allocate device memory when they launch work (an
allocator that owns the whole device, latency-critical loops where cudaMalloc
could synchronise the device, fixed memory budgets). For them the library keeps
the persistent batch kernel's counters in one fixed device array instead of
memory the batch allocated. These tests check, through the C ABI, that two such
launches in a row give the same fields as two launches of the regular entry
point (bit for bit: both run the same kernel on the same schedule), that they
leave the device's free memory unchanged, and that a batch larger than the
array's limit is refused.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import paper_2209_08437_gb300 as S
import sfac_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def problems():
    specs = [((32, 64), 3), ((512, 32), 2), ((128, 128), 4), ((64, 32, 32), 3), ((256, 64), 0), ((64, 64), 5)]
    out = []
    for k, (n, steps) in enumerate(specs):
        alpha = tuple(1.15 + 0.7 * I.uniform01(900 + k, len(n)))
        out.append(I.Problem(n=n, alpha=alpha, eps=0.05 + 0.02 * k, tau=2e-3, steps=steps))
    return out


@pytest.mark.parametrize("prec", [S.SFAC_FP64, S.SFAC_FP32])
def test_noalloc_launch_matches_regular_launch_twice(prec):
    probs = problems()
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    u0 = [I.random_field(p, 950 + k) for k, p in enumerate(probs)]
    regular = [torch.tensor(u, dtype=dt, device="cuda") for u in u0]
    noalloc = [torch.tensor(u, dtype=dt, device="cuda") for u in u0]
    steps = [p.steps for p in probs]
    lib = S.load()
    with S.Batch(probs, prec) as b:
        b.prepare(regular, steps)
        for _ in range(2):
            b.launch()
            b.wait()
        b.prepare(noalloc, steps)
        stream = torch.cuda.current_stream().cuda_stream
        assert lib.sfac_batch_launch_noalloc(b.handle, stream) == S.sfac.SFAC_OK  # set-up call
        b.wait()
        for k, u in enumerate(u0):
            noalloc[k].copy_(torch.tensor(u, dtype=dt))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        for _ in range(2):                      # two calls in a row through the C ABI
            assert lib.sfac_batch_launch_noalloc(b.handle, stream) == S.sfac.SFAC_OK
            b.wait()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before   # nothing was allocated
    for k in range(len(probs)):
        a = regular[k].cpu().numpy()
        c = noalloc[k].cpu().numpy()
        assert np.array_equal(a, c), k


def test_noalloc_refuses_batches_above_its_limit():
    p = I.Problem(n=(32, 32), alpha=(1.5, 1.5), eps=0.1, tau=1e-3)
    with S.Batch([p] * 8193, S.SFAC_FP32) as b:
        st = S.load().sfac_batch_launch_noalloc(b.handle, ctypes.c_void_p(0))
        assert st == S.sfac.SFAC_EINVAL
        assert "8192" in S.sfac_last_error()
