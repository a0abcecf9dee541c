"""Request loop over the sfac_server C ABI: continuous batching with admission
by device memory.

Requests arrive at their `arrival_s` times (scaled by `time_scale`, replayed
against the wall clock). Arrived requests are admitted in arrival order while
the server has a free slot and arena block (the library computes their FP64
tables and uploads field and tables). Each round advances every admitted request
by up to `chunk` steps in one persistent launch; a round is launched as soon as
the previous one has finished, and admission (host work) runs while it is on
the GPU, so requests admitted then join the next round. Finished requests are
copied back and their slots freed, which lets queued requests in. Latency is completion time
minus arrival time.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import sfac as _s


def serve(requests, make_u0, server: "_s.Server", chunk: int = 100, shape: int = 0,
          time_scale: float = 1.0, keep_results: bool = False, stream=None):
    """Serve `requests` (objects with rid, arrival_s, problem, problem.steps);
    make_u0(request) gives its initial field (numpy, server precision).
    Returns a dict with per-request latency, results (if kept) and totals."""
    dtype = np.float64 if server.prec == _s.SFAC_FP64 else np.float32
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival_s))
    queue = collections.deque()
    slot_req, latency, results = {}, {}, {}
    total_points = 0
    rounds = 0
    t0 = time.perf_counter()

    def now():
        return time.perf_counter() - t0

    def arrive():
        t = now()
        while pending and pending[0].arrival_s * time_scale <= t:
            queue.append(pending.popleft())

    def admit():
        while queue:
            r = queue[0]
            u0 = np.ascontiguousarray(make_u0(r), dtype=dtype)
            slot = server.admit(r.problem, u0, r.problem.steps)
            if slot is None:
                break
            slot_req[slot] = r
            queue.popleft()

    in_flight = False
    while pending or queue or slot_req:
        arrive()
        if not in_flight and slot_req:
            # the next round goes out first, so the GPU does not wait for admission
            server.round(chunk, shape, stream)
            rounds += 1
            in_flight = True
        admit()                                    # overlaps the round in flight, if any
        if in_flight:
            finished = server.wait(stream)
            in_flight = False
            for slot in finished:
                r = slot_req.pop(slot)
                out = np.empty(r.problem.shape, dtype=dtype) if keep_results else None
                server.fetch(slot, out)
                latency[r.rid] = now() - r.arrival_s * time_scale
                total_points += r.problem.points * r.problem.steps
                if keep_results:
                    results[r.rid] = out
            continue
        if not slot_req and pending:
            time.sleep(max(0.0, min(0.01, pending[0].arrival_s * time_scale - now())))
    wall = now()
    lat = np.array([latency[r.rid] for r in requests]) if requests else np.zeros(1)
    return {"latency": latency, "results": results, "wall_s": wall, "rounds": rounds,
            "point_steps": total_points, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "throughput": total_points / wall if wall > 0 else 0.0}
