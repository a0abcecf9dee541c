"""GPU tests of the batched persistent runner (sfac_batch_*): every instance of
a mixed batch against the CPU FP64 oracle, the same result alone and in the
mix, every autotuner shape, graph replay, and the bounded dependency wait."""
import concurrent.futures
import multiprocessing
import os

import numpy as np
import pytest

import paper_2209_08437_gb300 as S
import sfac_inputs as I
from oracle import sfac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def mixed_problems():
    """Uneven sizes, orders, eps and step counts; 2D and 3D."""
    out = []
    specs = [((32, 64), 3), ((512, 32), 5), ((128, 128), 7), ((256, 64), 2), ((64, 512), 4),
             ((32, 32, 32), 6), ((64, 32, 128), 3), ((256, 256), 1), ((128, 32, 64), 0), ((64, 64), 12)]
    for k, (n, steps) in enumerate(specs):
        u = I.uniform01(500 + k, 4)
        alpha = tuple(1.1 + 0.8 * I.uniform01(600 + k, len(n)))
        out.append(I.Problem(n=n, alpha=alpha, eps=0.02 + 0.18 * float(u[0]), tau=2e-3 * (1 + float(u[1])),
                             steps=steps))
    return out


def fields_for(problems, prec, seed0=700):
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    u0 = [I.random_field(p, seed0 + k) for k, p in enumerate(problems)]
    return u0, [torch.tensor(u, dtype=dt, device="cuda") for u in u0]


def run_batch(problems, prec, config=None, fields=None):
    u0, dev = fields if fields is not None else fields_for(problems, prec)
    with S.Batch(problems, prec) as b:
        if config is not None:
            S.sfac_batch_set_config(b.handle, config)
        b.step(dev, [p.steps for p in problems])
    torch.cuda.synchronize()
    return u0, [d.double().cpu().numpy() for d in dev]


def test_mixed_batch_fp64_matches_oracle():
    probs = mixed_problems()
    u0, got = run_batch(probs, S.SFAC_FP64)
    for k, p in enumerate(probs):
        ref = O.solve(p, u0[k], p.steps)
        err = np.abs(got[k] - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, (k, p.n, err)


def test_mixed_batch_fp32_error():
    probs = mixed_problems()
    u0, _ = fields_for(probs, S.SFAC_FP64)
    u32 = [np.asarray(u, np.float32).astype(np.float64) for u in u0]
    dev = [torch.tensor(u, dtype=torch.float32, device="cuda") for u in u32]
    _, got = run_batch(probs, S.SFAC_FP32, fields=(u32, dev))
    for k, p in enumerate(probs):
        ref = O.solve(p, u0[k], p.steps)
        assert np.abs(got[k] - ref).max() <= 1e-5, (k, p.n)


@pytest.mark.parametrize("prec", [S.SFAC_FP32, S.SFAC_FP64])
def test_alone_equals_in_the_mix(prec):
    """Each instance gives bit-identical results run alone and inside the mix."""
    probs = mixed_problems()
    _, mixed = run_batch(probs, prec)
    u0, _ = fields_for(probs, prec)
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    for k in (0, 1, 5, 9):
        alone = torch.tensor(u0[k], dtype=dt, device="cuda")
        with S.Batch([probs[k]], prec) as b:
            b.step([alone], [probs[k].steps])
        torch.cuda.synchronize()
        assert np.array_equal(alone.double().cpu().numpy(), mixed[k]), k


def test_batch_matches_single_plan_fp32():
    probs = [p for p in mixed_problems() if p.steps > 0]
    _, got = run_batch(probs, S.SFAC_FP32)
    u0, _ = fields_for(probs, S.SFAC_FP32)
    for k, p in enumerate(probs):
        with S.Plan.for_problem(p, S.SFAC_FP32) as plan:
            u = torch.tensor(u0[k], dtype=torch.float32, device="cuda")
            plan.step(u, p.steps)
            torch.cuda.synchronize()
        assert np.abs(u.double().cpu().numpy() - got[k]).max() <= 2e-6, k


def test_every_config_agrees():
    probs = mixed_problems()[:6]
    base = None
    for c in range(S.sfac_batch_num_configs()):
        u0, got = run_batch(probs, S.SFAC_FP32, config=c)
        if base is None:
            base = got
            refs = [O.solve(p, u0[k], p.steps) for k, p in enumerate(probs)]
        for k in range(len(probs)):
            assert np.abs(got[k] - refs[k]).max() <= 1e-5, (c, k)


def test_zero_steps_leave_field_untouched():
    probs = mixed_problems()
    u0, got = run_batch(probs, S.SFAC_FP64)
    k = [i for i, p in enumerate(probs) if p.steps == 0][0]
    assert np.array_equal(got[k], u0[k])


def test_autotune_then_run():
    probs = mixed_problems()
    u0, dev = fields_for(probs, S.SFAC_FP32)
    with S.Batch(probs, S.SFAC_FP32) as b:
        b.prepare(dev, [p.steps for p in probs])
        choice = b.autotune(max_steps=3)
        assert 0 <= choice < S.sfac_batch_num_configs()
        assert S.sfac_batch_get_config(b.handle)[0] == choice
        # autotuning leaves the fields alone
        for k in range(len(probs)):
            assert np.array_equal(dev[k].double().cpu().numpy(), np.asarray(u0[k], np.float32))
        b.launch()
        b.wait()
    for k, p in enumerate(probs):
        ref = O.solve(p, u0[k], p.steps)
        assert np.abs(dev[k].double().cpu().numpy() - ref).max() <= 1e-5


def test_graph_replay_equals_two_runs():
    probs = mixed_problems()[:5]
    u0, dev_a = fields_for(probs, S.SFAC_FP32)
    _, dev_b = fields_for(probs, S.SFAC_FP32)
    steps = [p.steps for p in probs]
    with S.Batch(probs, S.SFAC_FP32) as b:
        b.step(dev_a, steps)
        b.step(dev_a, steps)
        b.prepare(dev_b, steps)
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                b.launch(s)
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        b.wait()
    for k in range(len(probs)):
        assert torch.equal(dev_a[k], dev_b[k]), k


def test_bounded_wait_reports_timeout_and_recovers():
    """A dependency that is never satisfied ends the launch with SFAC_ETIMEOUT
    after a short bounded wait; the batch and the context stay usable."""
    probs = mixed_problems()[:4]
    u0, dev = fields_for(probs, S.SFAC_FP64)
    steps = [3] * len(probs)
    with S.Batch(probs, S.SFAC_FP64) as b:
        S.sfac_batch_set_wait_limit(b.handle, 2000, hold_instance=1)
        with pytest.raises(S.SfacError) as ei:
            b.step(dev, steps)
        assert ei.value.status == S.sfac.SFAC_ETIMEOUT
        S.sfac_batch_set_wait_limit(b.handle, 20_000_000, hold_instance=-1)
        fresh = [torch.tensor(u, dtype=torch.float64, device="cuda") for u in u0]
        b.step(fresh, steps)
    torch.cuda.synchronize()
    for k, p in enumerate(probs):
        ref = O.solve(p, u0[k], 3)
        assert np.abs(fresh[k].cpu().numpy() - ref).max() / np.abs(ref).max() <= 1e-12


def test_full_512_instance_workload_sampled():
    """The 512-instance batched workload (2D, n in {64..512}, 50-500 steps, FP32)
    in one launch. Every instance stays finite and within the maximum principle
    (Theorem 1: |u0| <= 0.9 keeps |u| <= 1); per size, the first instance, the
    one with the most steps and the one with the smallest eps are checked
    against the FP64 oracle (max-norm error <= 1e-5)."""
    inst = I.batched_instances()
    probs = [p for _, p in inst]
    u0 = [I.batched_u0(seed, p) for seed, p in inst]
    dev = [torch.tensor(np.asarray(u, np.float32), device="cuda") for u in u0]
    with S.Batch(probs, S.SFAC_FP32) as b:
        b.step(dev, [p.steps for p in probs])
    torch.cuda.synchronize()
    for k, d in enumerate(dev):
        assert bool(torch.isfinite(d).all()), k
        assert float(d.abs().max()) <= 1 + 1e-6, k
    picked = set()
    for n in sorted({p.n[0] for p in probs}):
        ks = [k for k, p in enumerate(probs) if p.n[0] == n]
        picked |= {ks[0], max(ks, key=lambda k: probs[k].steps), min(ks, key=lambda k: probs[k].eps)}
    # the oracle runs in parallel host processes (spawned: no fork after CUDA use)
    order = sorted(picked, key=lambda k: probs[k].n[0])
    ctx = multiprocessing.get_context("spawn")
    with concurrent.futures.ProcessPoolExecutor(max_workers=min(len(order), os.cpu_count() or 1),
                                                mp_context=ctx) as pool:
        refs = {k: pool.submit(O.solve, probs[k], u0[k], probs[k].steps, "two_level", "spectral") for k in order}
        refs = {k: f.result() for k, f in refs.items()}
    for k in order:
        p = probs[k]
        ref = refs[k]
        err = float(np.abs(dev[k].double().cpu().numpy() - ref).max())
        print(f"batched instance {k}: n={p.n[0]} steps={p.steps} eps={p.eps:.3f}: FP32 max-norm error {err:.3e}")
        assert err <= 1e-5
