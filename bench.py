#!/usr/bin/env python3
"""Benchmark of the two-level Strang splitting SFAC time step on GB300.

One bench "step" is one full time step of eq. (finalstrang): d fused axis
passes over the field, J^Q folded into the first load and the last store.
Default workload: 2D, n = 1024 per axis (1,048,576 unknowns), alpha = (1.3, 1.7),
eps = 0.05, tau = 1e-3, u0 = 0.9 sin(pi x) sin(pi y) + U(-0.05, 0.05) noise.

Prints ONE JSON line (rank 0). `value` is point-steps/s of the FP64 path with
the field resident in HBM; the FP32 path is measured the same way and
reported under "paths". Each timed step is preceded by an L2 flush (a 256 MiB
write) and timed alone with CUDA events on the launching stream.

  python bench.py [--steps K] [--warmup W] [--workload 2d1024|2d64|3d256|3d512]
  python bench.py --impl reference      # the CPU FP64 oracle on the host cores
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sfac_inputs as I  # noqa: E402

METRIC = "point-steps/s FP32 vs FP64 path at stated err vs oracle; served p50/p99 latency"
UNIT = "point-steps/s"

PROBE_3D512 = I.Problem(n=(512, 512, 512), alpha=(1.2, 1.5, 1.8), eps=0.08, tau=2e-3)

WORKLOADS = {
    "2d1024": dict(problem=I.CONFIG2, u0=I.config2_u0,
                   name="2D SFAC n=1024^2 (1,048,576 unknowns), alpha=(1.3,1.7), eps=0.05, tau=1e-3, "
                        "domain [-1,1]^2, u0=0.9 sin(pi x) sin(pi y)+U(-0.05,0.05) seed 1"),
    "2d64": dict(problem=I.CONFIG1, u0=I.config1_u0,
                 name="2D SFAC n=64^2, alpha=(1.5,1.5), eps=0.1, tau=0.01, u0~U[-0.9,0.9] seed 0"),
    "3d256": dict(problem=I.CONFIG3, u0=I.config3_u0,
                  name="3D SFAC n=256^3 (16,777,216 unknowns), alpha=(1.2,1.5,1.8), eps=0.08, tau=2e-3, "
                       "u0~U[-1,1] seed 2"),
    # HBM probe: fields of 0.5 GB (FP32) and 1.07 GB (FP64), far above the 129 MB L2.
    "3d512": dict(problem=PROBE_3D512, u0=lambda: I.random_field(PROBE_3D512, 2, -1.0, 1.0),
                  name="3D SFAC n=512^3 (134,217,728 unknowns; HBM probe), alpha=(1.2,1.5,1.8), eps=0.08, "
                       "tau=2e-3, u0~U[-1,1] seed 2"),
}

# Algorithmic work of one fused axis pass per real unknown: six complex FFTs of
# length n per pair of real lines at the conventional 5 n log2 n flops, plus the
# diagonal multiplies, the twist and the nonlinear flow: 15 log2 n + 10 flops;
# bytes: one read and one write of the field.
def pass_flops_per_point(n: int) -> float:
    return 15.0 * math.log2(n) + 10.0


# Nominal FP64 rate of GB300 (the FP64 units, not tensor cores) used as the
# ALU roofline of the FP64 passes; the FP32 passes use 2 flops x 128 lanes x
# 152 SMs x 2.07 GHz. HBM: the measured copy bandwidth.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 2 * 128 * 152 * 2.07e9 / 1e12

# DRAM bytes (read + write) per launch from ncu, keyed by (workload, precision,
# axis): the mean of dram__bytes_read.sum + dram__bytes_write.sum over the
# warm-up and timed launches of
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
#       --clock-control none -k regex:axis_pass -c 20|30 --csv
#       python bench.py --steps 2 --warmup 3 [--workload 3d256] --parity-steps 0 --no-cpu-baseline
# (profiles/axis_pass_dram_traffic.md). A key must be removed when its kernel changes.
NCU_TRAFFIC = {
    # 2d1024 FP64: -k regex:axis_pass -s 6 -c 2 (the two passes of the first timed step)
    ("2d1024", "f64", 0): 8592128, ("2d1024", "f64", 1): 8580864,
    ("2d1024", "f32", 0): 4284598, ("2d1024", "f32", 1): 4285513,
    ("3d256", "f32", 0): 72380342, ("3d256", "f32", 1): 75123309, ("3d256", "f32", 2): 75733504,
    # 3d512: -k regex:axis_pass -s 15 -c 15 (the FP64 single-pass timings and the FP32 warm-up steps)
    ("3d512", "f32", 0): 1008508672, ("3d512", "f32", 1): 1014830250, ("3d512", "f32", 2): 1014986837,
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu, self.proc, self.path = gpu_index, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (identity on one rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def aggregate_rate(points: int, steps: int, world: int, total_ms: float) -> float:
    """Whole-job point-steps/s: every rank advanced `points` unknowns `steps` times
    (weak scaling) and the job took the slowest rank's time."""
    return world * points * steps / (total_ms / 1e3)


def time_gpu_path(S, torch, problem, u0, prec, steps, warmup, flush):
    """Warm up, then time `steps` single steps, each one sfac_step call after an
    L2 flush, with CUDA events on the current stream. Then time every axis pass
    on its own (same J^Q modes as in the step), each after an L2 flush, for the
    roofline's kernel duration."""
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    d = problem.dim
    with S.Plan.for_problem(problem, prec) as plan:
        u = torch.tensor(u0, dtype=dt, device="cuda")
        modes = [(1 if ax == 0 else 0, 1 if ax == d - 1 else 0) for ax in range(d)]
        for _ in range(warmup):
            flush.zero_()
            plan.step(u, 1)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            plan.step(u, 1)
            e1.record(stream)
        torch.cuda.synchronize()
        step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        per_axis = []
        for ax in range(d):
            aev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for e0, e1 in aev:
                flush.zero_()
                e0.record(stream)
                plan.axis_pass(u, ax, *modes[ax])
                e1.record(stream)
            torch.cuda.synchronize()
            per_axis.append([e0.elapsed_time(e1) for e0, e1 in aev])
        ok = bool(torch.isfinite(u).all())
    return {"step_ms": step_ms, "axis_ms": per_axis, "finite": ok, "launches": 2 * steps * d}


def time_e2e(S, torch, problem, u0, prec, steps):
    """The public host-memory entry point: H2D copy, one step, D2H copy per step."""
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    host = torch.tensor(u0, dtype=dt).pin_memory()
    arr = host.numpy()
    with S.Plan.for_problem(problem, prec) as plan:
        plan.step_host(arr, 1)      # allocates the staging buffer
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            plan.step_host(arr, 1)
        el = time.perf_counter() - t0
    nbytes = arr.nbytes
    return {"value": problem.points * steps / el, "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}


def parity_check(S, torch, problem, u0, nsteps):
    """FP64 and FP32 paths against the CPU FP64 oracle after `nsteps` steps."""
    from oracle import sfac_oracle as O
    ref = O.solve(problem, u0, nsteps)
    out = {"steps": nsteps}
    for prec, key in ((S.SFAC_FP64, "f64_rel_err"), (S.SFAC_FP32, "f32_max_err")):
        dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
        with S.Plan.for_problem(problem, prec) as plan:
            u = torch.tensor(u0, dtype=dt, device="cuda")
            plan.step(u, nsteps)
            got = u.double().cpu().numpy()
        err = float(np.abs(got - ref).max())
        out[key] = err / float(np.abs(ref).max()) if prec == S.SFAC_FP64 else err
    return out


def cpu_baseline(problem, u0, budget_s=12.0):
    """The CPU FP64 oracle as it stands: dense per-axis factors (built once,
    not timed), then steps on the full grid until about budget_s seconds."""
    from oracle import sfac_oracle as O
    sch = O.Scheme.for_problem(problem)
    u = np.array(u0, dtype=np.float64)
    u = sch.step(u)
    steps, t0 = 0, time.perf_counter()
    while True:
        u = sch.step(u)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 100000:
            break
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    return {"value": problem.points * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} oracle steps on the full {'x'.join(map(str, problem.n))} grid "
                      f"({el:.1f} s; dense per-axis factors built beforehand, untimed; numpy/BLAS threads "
                      f"on all {cores} cores)"}


def run_batched(args, S, torch):
    """The 512-instance batched workload: one persistent launch advances every
    instance by its own step count; the launch is captured in a CUDA graph and
    each timed repetition replays it (inputs: 512 fields, ~178 MB of FP32, larger
    than L2)."""
    inst = I.batched_instances()
    probs = [p for _, p in inst]
    u0 = [I.batched_u0(seed, p) for seed, p in inst]
    steps = [p.steps for p in probs]
    work = sum(p.points * p.steps for p in probs)
    flops = sum(p.points * p.steps * sum(pass_flops_per_point(n) for n in p.n) for p in probs)
    dev = [torch.tensor(np.asarray(u, np.float32), device="cuda") for u in u0]
    batch = S.Batch(probs, S.SFAC_FP32)
    batch.prepare(dev, steps)
    choice = batch.autotune(max_steps=20)
    cfg = S.sfac_batch_get_config(batch.handle)
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            batch.launch(stream)
    for _ in range(max(args.warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()
    batch.wait()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    cur = torch.cuda.current_stream()
    for e0, e1 in evs:
        e0.record(cur)
        graph.replay()
        e1.record(cur)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    batch.wait()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = sum(ms)
    value = work * args.steps / (total_ms / 1e3)
    achieved = flops / (total_ms / args.steps / 1e3) / 1e12
    finite = all(bool(torch.isfinite(d).all()) for d in dev)
    # parity: fresh fields, one batch run, one instance per size against the oracle
    from oracle import sfac_oracle as O
    fresh = [torch.tensor(np.asarray(u, np.float32), device="cuda") for u in u0]
    batch.step(fresh, steps)
    torch.cuda.synchronize()
    picked = {}
    for k, p in enumerate(probs):
        picked.setdefault(p.n[0], k)
    errs = {}
    for n, k in sorted(picked.items()):
        if args.parity_steps <= 0:
            break
        ref = O.solve(probs[k], u0[k], steps[k], route="spectral")
        errs[str(n)] = float(np.abs(fresh[k].double().cpu().numpy() - ref).max())
    batch.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched: 512 independent 2D instances, n in {64,128,256,512}, alpha per axis "
                               "U[1.1,1.9], eps U[0.02,0.2], tau=1e-3, 50-500 steps each, FP32 with FP64 tables, "
                               "u0 U[-0.9,0.9], seeds 100-611; one persistent graph-captured launch per step",
                   "point_steps_per_run": work, "l2": "inputs (178 MB) larger than L2",
                   "autotuned_config": {"index": choice, "warps_per_cta": cfg[1], "values_per_thread": cfg[2],
                                        "groups_per_item": cfg[3]}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "batch_kernel<float>",
                     "kernel_ms": total_ms / args.steps,
                     "peak_source": "2 x 128 FP32 lanes x 152 SMs x 2.07 GHz"},
        "parity": {"f32_max_err_sampled": errs},
        "e2e": None, "cpu_baseline": None, "clocks": clocks, "gpu_launches": args.steps, "finite": finite,
    }
    print(json.dumps(line))
    return 0


def serving_shape(S, torch, sample, chunk):
    """Kernel shape for the serving rounds: the batch autotuner's choice on the
    first requests of the stream (their problems and initial fields, one round
    of `chunk` steps), measured before the timed region."""
    probs = [r.problem for r in sample]
    dev = [torch.tensor(np.asarray(I.request_u0(r), np.float32), device="cuda") for r in sample]
    with S.Batch(probs, S.SFAC_FP32) as b:
        b.prepare(dev, [min(p.steps, chunk) for p in probs])
        b.autotune(max_steps=chunk)
        cfg = S.sfac_batch_get_config(b.handle)
    del dev
    torch.cuda.empty_cache()
    return cfg


def run_serving(args, S, torch):
    """Poisson stream of 2000 requests (200/s; half 2D n in {64..512}, half 3D n in
    {32,64,128}; 100-1000 steps; FP32) served with continuous batching: requests
    are admitted by device memory into a 2 GiB arena and advanced in rounds of
    `chunk` steps by the persistent batch kernel."""
    reqs = I.serving_stream(args.requests)
    chunk = args.chunk
    S.load()
    cfg = serving_shape(S, torch, reqs[:64], chunk)
    shape = cfg[0]
    with S.Server(2 << 30, 1024, S.SFAC_FP32) as srv:
        # warm-up: a few small requests
        S.serve(I.serving_stream(8, rate_hz=1e6, sizes_2d=(64,), sizes_3d=(32,), steps_range=(5, 10)),
                lambda r: np.asarray(I.request_u0(r), np.float32), srv, chunk=chunk, shape=shape)
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        out = S.serve(reqs, lambda r: np.asarray(I.request_u0(r), np.float32), srv, chunk=chunk, shape=shape)
        clocks = sampler.stop()
    lat = np.array(list(out["latency"].values()))
    line = {
        "metric": METRIC, "value": out["throughput"], "unit": UNIT, "n_gpus": 1, "steps": out["rounds"],
        "warmup": 1, "ms_per_step": 1e3 * out["wall_s"] / max(out["rounds"], 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serving: Poisson stream of {len(reqs)} requests at 200/s, half 2D n in "
                               "{64,128,256,512}, half 3D n in {32,64,128}, alpha U[1.1,1.9], eps U[0.02,0.2], "
                               "tau=1e-3, 100-1000 steps, FP32; continuous batching in rounds of "
                               f"{chunk} steps, admission by a 2 GiB device arena",
                   "requests": len(reqs), "chunk_steps": chunk,
                   "kernel_shape": dict(zip(("index", "warps_per_cta", "values_per_thread", "groups_per_item"),
                                            cfg))},
        "latency": {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "mean_s": float(lat.mean()), "max_s": float(lat.max())},
        "served_point_steps": out["point_steps"], "wall_s": out["wall_s"], "rounds": out["rounds"],
        "clocks": clocks, "gpu_launches": out["rounds"],
    }
    print(json.dumps(line))
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    problem = w["problem"]
    u0 = w["u0"]()
    from oracle import sfac_oracle as O
    sch = O.Scheme.for_problem(problem)
    u = np.array(u0, dtype=np.float64)
    for _ in range(args.warmup):
        u = sch.step(u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = sch.step(u)
    el = time.perf_counter() - t0
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    value = problem.points * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed oracle steps on the full grid after "
                                       f"{args.warmup} warm-up steps (dense factors built beforehand)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sfac", choices=["sfac", "reference"])
    ap.add_argument("--workload", default="2d1024", choices=sorted(WORKLOADS) + ["batch512", "serve"])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--parity-steps", type=int, default=50)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2209_08437_gb300 as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if args.workload == "batch512":
        return run_batched(args, S, torch)
    if args.workload == "serve":
        return run_serving(args, S, torch)
    w = WORKLOADS[args.workload]
    problem = w["problem"]
    u0 = w["u0"]()
    S.load()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    r64 = time_gpu_path(S, torch, problem, u0, S.SFAC_FP64, args.steps, max(args.warmup, 3), flush)
    clocks = sampler.stop() if sampler else None
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    r32 = time_gpu_path(S, torch, problem, u0, S.SFAC_FP32, args.steps, max(args.warmup, 3), flush)

    t64, t32 = max_over_ranks([sum(r64["step_ms"]), sum(r32["step_ms"])], dist, "cuda")
    if rank != 0:
        dist.barrier() if dist else None
        return 0

    pts = problem.points
    d = problem.dim
    value64 = aggregate_rate(pts, args.steps, world, t64)
    value32 = aggregate_rate(pts, args.steps, world, t32)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)

    def roofline(res, prec_name, peak_tflops):
        axis_avg = [sum(a) / len(a) for a in res["axis_ms"]]
        ax = int(np.argmax(axis_avg))
        t = axis_avg[ax] / 1e3
        w_bytes = 8 if prec_name == "f64" else 4
        flops = pass_flops_per_point(problem.n[ax]) * pts
        bytes_ = 2 * w_bytes * pts
        gflops = flops / t / 1e12
        gbs = bytes_ / t / 1e9
        frac_alu = gflops / peak_tflops
        frac_hbm = gbs / hbm
        traffic = NCU_TRAFFIC.get((args.workload, prec_name, ax))
        if frac_alu >= frac_hbm:
            out = {"bound": "alu", "achieved": gflops, "peak": peak_tflops, "unit": "TFLOP/s",
                   "frac": frac_alu}
        else:
            out = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": frac_hbm}
        out.update({"traffic": traffic, "kernel": f"axis_pass axis {ax + 1} (n={problem.n[ax]})",
                    "kernel_ms": axis_avg[ax], "algorithmic_bytes": bytes_, "algorithmic_flops": flops,
                    "hbm_gbs": gbs, "hbm_frac_of_measured": frac_hbm,
                    "peak_source": ("nominal GB300 FP64 rate" if prec_name == "f64"
                                    else "2 x 128 FP32 lanes x 152 SMs x 2.07 GHz")
                    if out["bound"] == "alu" else "measured copy bandwidth (MEASURED_PEAKS.json)"})
        return out

    rf64 = roofline(r64, "f64", FP64_PEAK_TFLOPS)
    rf32 = roofline(r32, "f32", FP32_PEAK_TFLOPS)
    e2e = time_e2e(S, torch, problem, u0, S.SFAC_FP64, max(3, min(args.steps, 10)))
    e2e["value"] *= world
    parity = parity_check(S, torch, problem, u0, args.parity_steps) if args.parity_steps > 0 else None
    # the oracle's CPU baseline is timed at N = 1 only
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(problem, u0)

    line = {
        "metric": METRIC, "value": value64, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t64 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "points": pts, "dims": d,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": rf64,
        "paths": {"f64": {"value": value64, "ms_per_step": t64 / args.steps, "roofline": rf64},
                  "f32": {"value": value32, "ms_per_step": t32 / args.steps, "roofline": rf32,
                          "speedup_vs_f64": value32 / value64}},
        "parity": parity,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": r64["launches"],
        "finite": r64["finite"] and r32["finite"],
    }
    print(json.dumps(line))
    if dist:
        dist.barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
