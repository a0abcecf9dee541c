#!/usr/bin/env python3
"""Benchmark of the two-level Strang splitting SFAC time step on GB300.

One bench "step" is one full time step of eq. (finalstrang): d fused axis
passes over the field, J^Q folded into the first load and the last store.

Default run: the 3D workload, n = 256 per axis (16,777,216 unknowns),
alpha = (1.2, 1.5, 1.8), eps = 0.08, tau = 2e-3, u0 ~ U[-1, 1] from seed 2.
`value` is point-steps/s of the FP64 path with the field resident in HBM;
the FP32 path is measured the same way under "paths". Every timed step is
preceded by an L2 flush (a 256 MiB write) and timed alone with CUDA events on
the launching stream. The same line carries, under "workloads", the 2D
n = 1024 workload (FP64 and FP32), the 2D n = 64 workload's wall time (per step
and per 100-step run), the 512-instance batched workload and the served
Poisson request stream with its p50/p99 latency; and, under "peaks_measured",
the multiply-add rates that a probe kernel reaches on this GPU.

  python bench.py [--steps K] [--warmup W] [--workload 3d256|2d1024|2d64|3d512|2d4096|batch512|serve]
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
PROBE_2D4096 = I.Problem(n=(4096, 4096), alpha=(1.3, 1.7), eps=0.05, tau=1e-3)

WORKLOADS = {
    "3d256": dict(problem=I.CONFIG3, u0=I.config3_u0, parity_steps=3,
                  name="3D SFAC n=256^3 (16,777,216 unknowns), alpha=(1.2,1.5,1.8), eps=0.08, tau=2e-3, "
                       "domain [-1,1]^3, u0~U[-1,1] seed 2"),
    "2d1024": dict(problem=I.CONFIG2, u0=I.config2_u0, parity_steps=50,
                   name="2D SFAC n=1024^2 (1,048,576 unknowns), alpha=(1.3,1.7), eps=0.05, tau=1e-3, "
                        "domain [-1,1]^2, u0=0.9 sin(pi x) sin(pi y)+U(-0.05,0.05) seed 1"),
    "2d64": dict(problem=I.CONFIG1, u0=I.config1_u0, parity_steps=100,
                 name="2D SFAC n=64^2, alpha=(1.5,1.5), eps=0.1, tau=0.01, domain [-1,1]^2, "
                      "u0~U[-0.9,0.9] seed 0"),
    # HBM probe: fields of 0.5 GB (FP32) and 1.07 GB (FP64), far above the 129 MB L2.
    "3d512": dict(problem=PROBE_3D512, u0=lambda: I.random_field(PROBE_3D512, 2, -1.0, 1.0), parity_steps=0,
                  name="3D SFAC n=512^3 (134,217,728 unknowns; HBM probe), alpha=(1.2,1.5,1.8), eps=0.08, "
                       "tau=2e-3, u0~U[-1,1] seed 2"),
    # Long lines: 4096-point FFTs (radix 16), fields of 67 MB (FP32) and 134 MB (FP64).
    "2d4096": dict(problem=PROBE_2D4096, u0=lambda: I.random_field(PROBE_2D4096, 1, -0.9, 0.9), parity_steps=0,
                   name="2D SFAC n=4096^2 (16,777,216 unknowns; long-line probe), alpha=(1.3,1.7), eps=0.05, "
                        "tau=1e-3, u0~U[-0.9,0.9] seed 1"),
}


# Algorithmic work of one fused axis pass per real unknown: six complex FFTs of
# length n per pair of real lines at the conventional 5 n log2 n flops, plus the
# diagonal multiplies, the twist and the nonlinear flow: 15 log2 n + 10 flops;
# bytes: one read and one write of the field.
def pass_flops_per_point(n: int) -> float:
    return 15.0 * math.log2(n) + 10.0


# ALU rooflines, derived from unit counts and the 2.07 GHz maximum SM clock:
# FP64 2 fma/clk/SM x 152 SMs x 2 flops (1.25 TFLOP/s, the nominal GB300 FP64
# rate); FP32 128 lanes x 152 SMs x 2 flops. The probe kernel's measured rates
# are reported beside them.
SM_CLOCK_GHZ = 2.07
FP64_PEAK_TFLOPS = 2 * 152 * 2 * SM_CLOCK_GHZ / 1e3
FP32_PEAK_TFLOPS = 128 * 152 * 2 * SM_CLOCK_GHZ / 1e3
PEAK_SOURCE = {"f64": "derived: 2 FP64 fma/clk/SM x 152 SMs x 2 flops x 2.07 GHz",
               "f32": "derived: 128 FP32 lanes x 152 SMs x 2 flops x 2.07 GHz"}

# DRAM bytes (read + write) per launch from ncu, keyed by (workload, precision,
# axis): the mean of dram__bytes_read.sum + dram__bytes_write.sum over the
# captured launches of each pass, from
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum --clock-control none
#       -k regex:axis_pass [-s 15] -c <launches>
#       python bench.py --workload <w> --steps 2 --warmup 3 --parity-steps 0 --no-cpu-baseline --no-extras
# (-c 28 for 2d1024 and 2d4096, -c 42 for 3d256, -s 15 -c 15 for 3d512). An entry is
# removed when its kernel changes.
NCU_TRAFFIC = {
    ("2d1024", "f64", 0): 8570000, ("2d1024", "f64", 1): 8585714,
    ("2d1024", "f32", 0): 4281429, ("2d1024", "f32", 1): 4291429,
    ("3d256", "f64", 0): 203777143, ("3d256", "f64", 1): 209997143, ("3d256", "f64", 2): 209608571,
    ("3d256", "f32", 0): 72635714, ("3d256", "f32", 1): 75765714, ("3d256", "f32", 2): 75717143,
    ("3d512", "f64", 0): 2085800000, ("3d512", "f64", 1): 2090875000, ("3d512", "f64", 2): 2091510000,
    ("3d512", "f32", 0): 1008836667, ("3d512", "f32", 1): 1014696667, ("3d512", "f32", 2): 1014876667,
    ("2d4096", "f64", 0): 205950000, ("2d4096", "f64", 1): 213458571,
    ("2d4096", "f32", 0): 71625714, ("2d4096", "f32", 1): 78167143,
}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons. Sampling runs only
    between start() and stop(); several such segments (the timed regions) are
    pooled into one summary()."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu, self.proc, self.path, self.rows = gpu_index, None, None, []

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)  # nvidia-smi's own start-up, so that the segment is sampled from its start
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    self.rows.append(parts)
        finally:
            os.unlink(self.path)
        self.proc = None

    def summary(self):
        rows = self.rows
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
    return {"step_ms": step_ms, "axis_ms": per_axis, "finite": ok, "launches": steps * d}


HOST_ROUTES = {0: "copy: cudaMemcpyAsync in and out around the step",
               1: "mapped: the first pass loads the field from the pinned host buffer over NVLink-C2C, "
                  "the last pass stores the result into it",
               2: "mapped in: the first pass loads the field from the pinned host buffer, a copy brings "
                  "the result back"}


def time_e2e(S, torch, problem, u0, prec, steps):
    """The public host-memory entry point, one step per call: the field moves
    from pinned host memory to the GPU and the result back in every call."""
    dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
    host = torch.tensor(u0, dtype=dt).pin_memory()
    arr = host.numpy()
    with S.Plan.for_problem(problem, prec) as plan:
        route = plan.host_route(arr, 1)
        plan.step_host(arr, 1)      # allocates the staging buffer
        torch.cuda.synchronize()
        # three blocks of `steps` calls; the median block is reported (the
        # host and its link are shared, and one block once ran 2.7x slow)
        blocks = []
        for _ in range(3):
            t0 = time.perf_counter()
            for _ in range(steps):
                plan.step_host(arr, 1)
            blocks.append(time.perf_counter() - t0)
        el = sorted(blocks)[1]
    nbytes = arr.nbytes
    # The host link's own rate, for the bound it puts on this number: one
    # pinned-host-to-device and one device-to-pinned-host copy of the field
    # (cudaMemcpyAsync through torch), best of three each.
    dev = torch.empty_like(host, device="cuda")
    rates = {}
    for name, src, dst in (("h2d", host, dev), ("d2h", dev, host)):
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dst.copy_(src, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        rates[name] = nbytes / best / 1e9
    link_s = nbytes / (rates["h2d"] * 1e9) + nbytes / (rates["d2h"] * 1e9)
    return {"value": problem.points * steps / el, "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "call": "sfac_step_host(plan, pinned host field, 1)", "route": HOST_ROUTES.get(route, str(route)),
            "blocks_s": blocks, "calls_per_block": steps,
            "link_gbs": {"h2d": rates["h2d"], "d2h": rates["d2h"]},
            "link_bound": problem.points / link_s}


def roofline(workload, problem, res, prec_name, peaks_live):
    """Roofline record of the slowest axis pass of one path."""
    pts = problem.points
    axis_avg = [sum(a) / len(a) for a in res["axis_ms"]]
    ax = int(np.argmax(axis_avg))
    t = axis_avg[ax] / 1e3
    w_bytes = 8 if prec_name == "f64" else 4
    flops = pass_flops_per_point(problem.n[ax]) * pts
    bytes_ = 2 * w_bytes * pts
    tflops = flops / t / 1e12
    gbs = bytes_ / t / 1e9
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    peak = FP64_PEAK_TFLOPS if prec_name == "f64" else FP32_PEAK_TFLOPS
    frac_alu, frac_hbm = tflops / peak, gbs / hbm
    if frac_alu >= frac_hbm:
        out = {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": frac_alu}
        live = (peaks_live or {}).get("fp64_tflops" if prec_name == "f64" else "fp32_tflops")
        src = PEAK_SOURCE[prec_name]
        if live:
            out.update({"peak_measured": live, "frac_of_measured": tflops / live})
            src += f"; the fma probe measured {live:.3g} TFLOP/s in this run"
        out["peak_source"] = src
    else:
        out = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": frac_hbm,
               "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"}
    out.update({"traffic": NCU_TRAFFIC.get((workload, prec_name, ax)),
                "kernel": f"axis_pass axis {ax + 1} (n={problem.n[ax]})", "kernel_ms": axis_avg[ax],
                "per_axis_ms": axis_avg, "algorithmic_bytes": bytes_, "algorithmic_flops": flops,
                "hbm_gbs": gbs, "hbm_frac_of_measured": frac_hbm})
    return out


def measure_grid(S, torch, key, steps, warmup, flush, peaks_live, e2e=True, world=1, dist=None):
    """FP64 and FP32 paths of one single-grid workload."""
    w = WORKLOADS[key]
    problem = w["problem"]
    u0 = w["u0"]()
    r64 = time_gpu_path(S, torch, problem, u0, S.SFAC_FP64, steps, warmup, flush)
    r32 = time_gpu_path(S, torch, problem, u0, S.SFAC_FP32, steps, warmup, flush)
    t64, t32 = max_over_ranks([sum(r64["step_ms"]), sum(r32["step_ms"])], dist, "cuda")
    v64 = aggregate_rate(problem.points, steps, world, t64)
    v32 = aggregate_rate(problem.points, steps, world, t32)
    out = {
        "workload": w["name"], "points": problem.points, "steps": steps, "warmup": warmup,
        "f64": {"value": v64, "ms_per_step": t64 / steps, "roofline": roofline(key, problem, r64, "f64", peaks_live),
                "gpu_launches": r64["launches"]},
        "f32": {"value": v32, "ms_per_step": t32 / steps, "roofline": roofline(key, problem, r32, "f32", peaks_live),
                "gpu_launches": r32["launches"], "speedup_vs_f64": v32 / v64},
        "finite": r64["finite"] and r32["finite"],
    }
    if e2e:
        n_e2e = max(3, min(steps, 10))
        out["f64"]["e2e"] = time_e2e(S, torch, problem, u0, S.SFAC_FP64, n_e2e)
        out["f32"]["e2e"] = time_e2e(S, torch, problem, u0, S.SFAC_FP32, n_e2e)
        for p in ("f64", "f32"):
            out[p]["e2e"]["value"] *= world
    return out


def measure_small_grid(S, torch, steps, warmup, flush):
    """The 2D n = 64 workload (a 32 KB field): wall time of one step and of a
    whole 100-step run, for both paths, launched directly and as a replayed
    CUDA graph of the 100-step call. Each timed call follows an L2 flush."""
    w = WORKLOADS["2d64"]
    problem = w["problem"]
    u0 = w["u0"]()
    nrun = problem.steps
    stream = torch.cuda.current_stream()
    out = {"workload": w["name"], "points": problem.points, "run_steps": nrun}

    def timed(fn, reps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    for prec, name in ((S.SFAC_FP64, "f64"), (S.SFAC_FP32, "f32")):
        dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
        with S.Plan.for_problem(problem, prec) as plan:
            u = torch.tensor(u0, dtype=dt, device="cuda")
            for _ in range(warmup):
                plan.step(u, 1)
                plan.step(u, nrun)
            torch.cuda.synchronize()
            step_ms = timed(lambda: plan.step(u, 1), steps)
            run_ms = timed(lambda: plan.step(u, nrun), max(3, steps // 4))
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                with torch.cuda.graph(graph, stream=side):
                    plan.step(u, nrun, stream=side.cuda_stream)
            stream.wait_stream(side)
            for _ in range(warmup):
                graph.replay()
            torch.cuda.synchronize()
            graph_ms = timed(graph.replay, max(3, steps // 4))
            del graph
            whole = plan.step_kernel(nrun) == S.SFAC_STEP_WHOLE
        best = min(statistics.median(run_ms), statistics.median(graph_ms))
        out[name] = {"ms_per_step_single_call": statistics.median(step_ms),
                     "ms_per_run": statistics.median(run_ms), "ms_per_run_graph": statistics.median(graph_ms),
                     "value": problem.points * nrun / (best / 1e3),
                     "whole_call_launch": whole,
                     "gpu_launches_per_run": 1 if whole else nrun * problem.dim}
    return out


def measure_probe(S, torch):
    """Multiply-add rates of the probe kernel (best of 3 launches each):
    8 CTAs of 256 threads per SM, 8 independent chains per thread."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks = 8 * sms
    stream = torch.cuda.current_stream()
    out = {"blocks": blocks, "threads": 256}
    for kind, key, iters in ((0, "fp64_tflops", 250), (1, "fp32_tflops", 12000), (2, "fp32_packed_tflops", 6000)):
        buf = torch.empty(blocks * 256, dtype=torch.float64 if kind == 0 else torch.float32, device="cuda")
        S.sfac.sfac_probe_fma(kind, blocks, 4, buf)  # warm-up
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flops = S.sfac.sfac_probe_fma(kind, blocks, iters, buf)
            e1.record(stream)
            torch.cuda.synchronize()
            rate = flops / (e0.elapsed_time(e1) / 1e3) / 1e12
            best = rate if best is None else max(best, rate)
        out[key] = best
    return out


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


def full_run_parity(S, torch, key, problem, u0):
    """The whole run of the 3D workload (500 steps, one sfac_step call per
    path) against the oracle's field stored at 4096 points
    (tests/golden/config3_oracle_spectral_500.txt, written from oracle/ only),
    and the FP32 field against the FP64 one everywhere."""
    if key != "3d256":
        return None
    path = os.path.join(ROOT, "tests", "golden", "config3_oracle_spectral_500.txt")
    if not os.path.exists(path):
        return None
    idx, val, max_abs = [], [], None
    for line in open(path):
        if line.startswith("# max_abs"):
            max_abs = float(line.split()[2])
        elif line.strip() and not line.startswith("#"):
            i, v = line.split()
            idx.append(int(i))
            val.append(float(v))
    idx, val = np.array(idx), np.array(val)
    out = {"steps": problem.steps, "reference": "oracle (spectral route) at 4096 stored points"}
    fields = {}
    for prec, name in ((S.SFAC_FP64, "f64"), (S.SFAC_FP32, "f32")):
        dt = torch.float64 if prec == S.SFAC_FP64 else torch.float32
        with S.Plan.for_problem(problem, prec) as plan:
            u = torch.tensor(u0, dtype=dt, device="cuda")
            plan.step(u, problem.steps)
            plan.check()
            fields[name] = u.double()
    f64 = fields["f64"].reshape(-1).cpu().numpy()
    f32 = fields["f32"].reshape(-1).cpu().numpy()
    out["f64_rel_err"] = float(np.abs(f64[idx] - val).max()) / max_abs
    out["f32_max_err"] = float(np.abs(f32[idx] - val).max())
    out["f32_vs_f64_full_field"] = float((fields["f32"] - fields["f64"]).abs().max())
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
    cores = host_cores()
    grid = "x".join(map(str, problem.n))
    sample = (f"{steps} oracle steps on the full {grid} grid ({el:.1f} s; dense per-axis factors built "
              f"beforehand, untimed; numpy/BLAS threads on all {cores} cores)")
    if problem.steps > steps:
        sample += (f"; the full {problem.steps}-step run extrapolates linearly to "
                   f"{el / steps * problem.steps:.0f} s")
    return {"value": problem.points * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}


def measure_batched(S, torch, steps, warmup, parity_steps=0):
    """The 512-instance batched workload: one persistent launch advances every
    instance by its own step count; the launch is captured in a CUDA graph and
    each timed repetition replays it (inputs: 512 fields, ~178 MB of FP32, larger
    than L2)."""
    inst = I.batched_instances()
    probs = [p for _, p in inst]
    u0 = [I.batched_u0(seed, p) for seed, p in inst]
    nsteps = [p.steps for p in probs]
    work = sum(p.points * p.steps for p in probs)
    flops = sum(p.points * p.steps * sum(pass_flops_per_point(n) for n in p.n) for p in probs)
    dev = [torch.tensor(np.asarray(u, np.float32), device="cuda") for u in u0]
    batch = S.Batch(probs, S.SFAC_FP32)
    batch.prepare(dev, nsteps)
    choice = batch.autotune(max_steps=20)
    cfg = S.sfac_batch_get_config(batch.handle)
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            batch.launch(stream)
    for _ in range(max(warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()
    batch.wait()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    cur = torch.cuda.current_stream()
    for e0, e1 in evs:
        e0.record(cur)
        graph.replay()
        e1.record(cur)
    torch.cuda.synchronize()
    batch.wait()
    ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = sum(ms)
    achieved = flops / (total_ms / steps / 1e3) / 1e12
    finite = all(bool(torch.isfinite(d).all()) for d in dev)
    errs = {}
    if parity_steps > 0:
        # fresh fields, one batch run, one instance per size against the oracle
        from oracle import sfac_oracle as O
        fresh = [torch.tensor(np.asarray(u, np.float32), device="cuda") for u in u0]
        batch.step(fresh, nsteps)
        torch.cuda.synchronize()
        picked = {}
        for k, p in enumerate(probs):
            picked.setdefault(p.n[0], k)
        for n, k in sorted(picked.items()):
            ref = O.solve(probs[k], u0[k], nsteps[k], route="spectral")
            errs[str(n)] = float(np.abs(fresh[k].double().cpu().numpy() - ref).max())
    batch.close()
    return {
        "workload": "batched: 512 independent 2D instances, n in {64,128,256,512}, alpha per axis U[1.1,1.9], "
                    "eps U[0.02,0.2], tau=1e-3, 50-500 steps each, FP32 with FP64 tables, u0 U[-0.9,0.9], "
                    "seeds 100-611; one persistent graph-captured launch per repetition",
        "value": work * steps / (total_ms / 1e3), "unit": UNIT, "dtype": "f32", "repetitions": steps,
        "ms_per_run": total_ms / steps, "point_steps_per_run": work, "l2": "inputs (178 MB) larger than L2",
        "autotuned_config": {"index": choice, "warps_per_cta": cfg[1], "values_per_thread": cfg[2],
                             "groups_per_item": cfg[3]},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "batch_kernel<float>",
                     "kernel_ms": total_ms / steps, "peak_source": PEAK_SOURCE["f32"]},
        "parity": {"f32_max_err_sampled": errs} if errs else None,
        "gpu_launches": steps, "finite": finite,
    }


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


def serving_samples(reqs):
    """Request ids whose results are checked against the oracle: the first
    request of each of 2D n = 64, 128, 256 and 3D n = 32, 64 (sizes the dense
    oracle finishes in seconds)."""
    want = {(2, 64), (2, 128), (2, 256), (3, 32), (3, 64)}
    picked = {}
    for r in reqs:
        key = (r.problem.dim, r.problem.n[0])
        if key in want and key not in picked:
            picked[key] = r.rid
    return picked


def measure_serving(S, torch, requests, chunk, sampler=None, check=True, max_in_flight=2):
    """Poisson stream of requests (200/s; half 2D n in {64..512}, half 3D n in
    {32,64,128}; 100-1000 steps; FP32) served with continuous batching: requests
    are admitted by device memory into a 2 GiB arena and advanced in rounds of
    `chunk` steps by the persistent batch kernel."""
    reqs = I.serving_stream(requests)
    cfg = serving_shape(S, torch, reqs[:64], chunk)
    shape = cfg[0]
    picked = serving_samples(reqs) if check else {}
    make = lambda r: np.asarray(I.request_u0(r), np.float32)  # noqa: E731
    pair = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))  # noqa: E731
    with S.Server(2 << 30, 1024, S.SFAC_FP32) as srv:
        # warm-up: a few small requests
        S.serve(I.serving_stream(8, rate_hz=1e6, sizes_2d=(64,), sizes_3d=(32,), steps_range=(5, 10)),
                make, srv, chunk=chunk, shape=shape)
        if sampler:
            sampler.start()
        out = S.serve(reqs, make, srv, chunk=chunk, shape=shape, keep_results=set(picked.values()),
                      round_events=pair, max_in_flight=max_in_flight)
        if sampler:
            sampler.stop()
    lat = np.array(list(out["latency"].values()))
    errs = {}
    if picked:
        from oracle import sfac_oracle as O
        for (dim, n), rid in sorted(picked.items()):
            r = reqs[rid]
            u0 = np.asarray(I.request_u0(r), np.float32).astype(np.float64)
            ref = O.solve(r.problem, u0, r.problem.steps)
            errs[f"{dim}d_n{n}_rid{rid}_{r.problem.steps}steps"] = float(np.abs(out["results"][rid] - ref).max())
    busy, span = out.get("gpu_busy_s"), out.get("gpu_span_s")
    return {
        "workload": f"serving: Poisson stream of {len(reqs)} requests at 200/s, half 2D n in {{64,128,256,512}}, "
                    "half 3D n in {32,64,128}, alpha U[1.1,1.9], eps U[0.02,0.2], tau=1e-3, 100-1000 steps, FP32; "
                    f"continuous batching in rounds of {chunk} steps, admission by a 2 GiB device arena",
        "value": out["throughput"], "unit": UNIT, "dtype": "f32", "requests": len(reqs), "chunk_steps": chunk,
        "rounds_in_flight": max_in_flight, "failed_requests": len(out["failed"]),
        "kernel_shape": dict(zip(("index", "warps_per_cta", "values_per_thread", "groups_per_item"), cfg)),
        "latency": {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "mean_s": float(lat.mean()), "max_s": float(lat.max())},
        "served_point_steps": out["point_steps"], "wall_s": out["wall_s"], "rounds": out["rounds"],
        "gpu_busy_s": busy, "gpu_span_s": span,
        "gpu_idle_frac": (1.0 - busy / span) if busy and span else None,
        "parity": {"f32_max_err_vs_fp64_oracle": errs} if errs else None,
        "gpu_launches": out["rounds"],
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    key = args.workload if args.workload in WORKLOADS else "3d256"
    w = WORKLOADS[key]
    problem = w["problem"]
    u0 = w["u0"]()
    from oracle import sfac_oracle as O
    sch = O.Scheme.for_problem(problem)
    u = np.array(u0, dtype=np.float64)
    # each step is a bounded sample of the workload: the dense route on the
    # full grid costs O(n^(d+1)) per step
    for _ in range(args.warmup):
        u = sch.step(u)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = sch.step(u)
    el = time.perf_counter() - t0
    cores = host_cores()
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
    ap.add_argument("--workload", default="3d256", choices=sorted(WORKLOADS) + ["batch512", "serve"])
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--max-in-flight", type=int, default=2, choices=[1, 2], help="serving rounds kept enqueued")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads and the probe")
    ap.add_argument("--parity-steps", type=int, default=None)
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
    S.load()
    warmup = max(args.warmup, 3)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None

    if args.workload in ("batch512", "serve"):
        if args.workload == "batch512":
            if sampler:
                sampler.start()
            rec = measure_batched(S, torch, args.steps, warmup, args.parity_steps or 0)
            if sampler:
                sampler.stop()
        else:
            rec = measure_serving(S, torch, args.requests, args.chunk, sampler,
                                  check=(args.parity_steps is None or args.parity_steps > 0),
                                  max_in_flight=args.max_in_flight)
        line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": 1,
                "steps": rec.get("repetitions", rec.get("rounds")), "warmup": warmup,
                "ms_per_step": rec.get("ms_per_run", 1e3 * rec.get("wall_s", 0) / max(rec.get("rounds", 1), 1)),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": {"workload": rec["workload"]}, "record": rec,
                "clocks": sampler.summary() if sampler else None, "gpu_launches": rec["gpu_launches"]}
        print(json.dumps(line))
        return 0

    key = args.workload
    w = WORKLOADS[key]
    problem = w["problem"]
    u0 = w["u0"]()
    parity_steps = w["parity_steps"] if args.parity_steps is None else args.parity_steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    extras = not args.no_extras and world == 1

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    peaks_live = measure_probe(S, torch) if extras else None
    head = measure_grid(S, torch, key, args.steps, warmup, flush, peaks_live, e2e=True, world=world, dist=dist)
    workloads = {}
    if extras:
        for k2 in ("2d1024", "3d256"):
            if k2 != key:
                workloads[k2] = measure_grid(S, torch, k2, args.steps, warmup, flush, peaks_live, e2e=False)
        workloads["2d64"] = measure_small_grid(S, torch, args.steps, warmup, flush)
        workloads["batched"] = measure_batched(S, torch, args.steps, warmup)
    if sampler:
        sampler.stop()
    if extras:
        workloads["serving"] = measure_serving(S, torch, args.requests, args.chunk, sampler,
                                               max_in_flight=args.max_in_flight)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    if rank != 0:
        return 0

    parity = parity_check(S, torch, problem, u0, parity_steps) if parity_steps > 0 else None
    if parity is not None and extras:
        parity["full_run"] = full_run_parity(S, torch, key, problem, u0)
    # the oracle's CPU baseline is timed at N = 1 only
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(problem, u0)
    f64, f32 = head["f64"], head["f32"]
    line = {
        "metric": METRIC, "value": f64["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": f64["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "points": problem.points, "dims": problem.dim,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": f64["roofline"],
        "paths": {"f64": f64, "f32": f32},
        "parity": parity,
        "e2e": f64["e2e"],
        "cpu_baseline": cpu,
        "clocks": sampler.summary() if sampler else None,
        "gpu_launches": f64["gpu_launches"],
        "peaks_measured": peaks_live,
        "workloads": workloads or None,
        "finite": head["finite"],
    }
    print(json.dumps(line))
    if dist:
        dist.barrier()
    return 0


if __name__ == "__main__":
    sys.exit(main())
