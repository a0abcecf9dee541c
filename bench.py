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

  python bench.py [--steps K] [--warmup W] [--workload 2d1024|2d64|3d256]
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

WORKLOADS = {
    "2d1024": dict(problem=I.CONFIG2, u0=I.config2_u0,
                   name="2D SFAC n=1024^2 (1,048,576 unknowns), alpha=(1.3,1.7), eps=0.05, tau=1e-3, "
                        "domain [-1,1]^2, u0=0.9 sin(pi x) sin(pi y)+U(-0.05,0.05) seed 1"),
    "2d64": dict(problem=I.CONFIG1, u0=I.config1_u0,
                 name="2D SFAC n=64^2, alpha=(1.5,1.5), eps=0.1, tau=0.01, u0~U[-0.9,0.9] seed 0"),
    "3d256": dict(problem=I.CONFIG3, u0=I.config3_u0,
                  name="3D SFAC n=256^3 (16,777,216 unknowns), alpha=(1.2,1.5,1.8), eps=0.08, tau=2e-3, "
                       "u0~U[-1,1] seed 2"),
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
# axis). None until a capture of the current kernels exists.
NCU_TRAFFIC = {}


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


def time_gpu_path(S, torch, problem, u0, prec, steps, warmup, flush):
    """Warm up, then time `steps` single steps (each after an L2 flush) as the
    sequence of its axis passes with CUDA events on the current stream."""
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    d = problem.dim
    with S.Plan.for_problem(problem, prec) as plan:
        u = torch.tensor(u0, dtype=dt, device="cuda")
        modes = [(1 if ax == 0 else 0, 1 if ax == d - 1 else 0) for ax in range(d)]

        def one_step():
            for ax in range(d):
                plan.axis_pass(u, ax, *modes[ax])

        for _ in range(warmup):
            flush.zero_()
            one_step()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(d + 1)] for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            for ax in range(d):
                plan.axis_pass(u, ax, *modes[ax])
                evs[k][ax + 1].record(stream)
        torch.cuda.synchronize()
        per_axis = [[evs[k][ax].elapsed_time(evs[k][ax + 1]) for k in range(steps)] for ax in range(d)]
        step_ms = [evs[k][0].elapsed_time(evs[k][d]) for k in range(steps)]
        ok = bool(torch.isfinite(u).all())
    return {"step_ms": step_ms, "axis_ms": per_axis, "finite": ok, "launches": steps * d}


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
    ap.add_argument("--workload", default="2d1024", choices=sorted(WORKLOADS))
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

    t64 = sum(r64["step_ms"])
    t32 = sum(r32["step_ms"])
    if dist:
        tt = torch.tensor([t64, t32], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t64, t32 = float(tt[0]), float(tt[1])
    if rank != 0:
        dist.barrier() if dist else None
        return 0

    pts = problem.points
    d = problem.dim
    value64 = world * pts * args.steps / (t64 / 1e3)
    value32 = world * pts * args.steps / (t32 / 1e3)
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
    cpu = None if args.no_cpu_baseline else cpu_baseline(problem, u0)

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
