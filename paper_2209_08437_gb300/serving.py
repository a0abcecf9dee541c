"""Request loop over the sfac_server C ABI: continuous batching with admission
by device memory.

Requests arrive at their `arrival_s` times (scaled by `time_scale`, replayed
against the wall clock). Arrived requests are admitted in arrival order while
the server has a free slot and arena block (the library computes their FP64
tables and uploads field and tables). Each round advances every admitted request
by up to `chunk` steps in one persistent launch. Up to `max_in_flight` rounds
are kept enqueued (the server allows two): the next round goes out behind the
one running, so the device does not wait while the host collects results, and
admission (host work) runs while rounds are on the GPU; requests admitted then
join a later round. Finished requests are copied back and their slots freed,
which lets queued requests in. Latency is completion time minus arrival time.
A request whose round gave up (the server's bounded waits) is reported under
"failed" and has no result; one that does not fit the server even when it
holds nothing else is reported under "rejected".
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import sfac as _s


def serve(requests, make_u0, server: "_s.Server", chunk: int = 100, shape: int = 0,
          time_scale: float = 1.0, keep_results=False, stream=None, round_events=None,
          max_in_flight: int = 2):
    """Serve `requests` (objects with rid, arrival_s, problem, problem.steps);
    make_u0(request) gives its initial field (numpy, server precision).
    keep_results: True keeps every result, a collection of request ids keeps
    those. round_events: optional factory of a (start, end) pair of CUDA events
    recorded around each round launch on the round's stream (anything with
    record() and elapsed_time()); the device time of the rounds is then
    reported as gpu_busy_s and the span from the first round's start to the last
    round's end as gpu_span_s.
    Returns a dict with per-request latency, results (if kept) and totals."""
    keep = (lambda rid: True) if keep_results is True else (
        (lambda rid: False) if not keep_results else (lambda rid, ids=frozenset(keep_results): rid in ids))
    evs = []
    failed, rejected = [], []
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
                if not slot_req:
                    # the server holds nothing (so no round is in flight) and the
                    # request still does not fit: it never will
                    rejected.append(queue.popleft().rid)
                    continue
                break
            slot_req[slot] = r
            queue.popleft()
            if r.problem.steps == 0:               # no round will hold it: done at once
                finish(slot)

    def finish(slot):
        nonlocal total_points
        r = slot_req.pop(slot)
        out = np.empty(r.problem.shape, dtype=dtype) if keep(r.rid) else None
        try:
            server.fetch(slot, out)
        except _s.SfacError as e:
            if e.status != _s.SFAC_ETIMEOUT:
                raise
            failed.append(r.rid)                   # its round gave up: no result
            return
        latency[r.rid] = now() - r.arrival_s * time_scale
        total_points += r.problem.points * r.problem.steps
        if out is not None:
            results[r.rid] = out

    in_flight = 0
    while pending or queue or slot_req:
        arrive()
        # the next rounds go out first, so the GPU does not wait for admission
        while in_flight < max_in_flight and slot_req:
            if round_events is not None:
                e0, e1 = round_events()
                e0.record()
            if not server.round(chunk, shape, stream):
                break                              # every active slot is covered by a round in flight
            if round_events is not None:
                e1.record()
                evs.append((e0, e1))
            rounds += 1
            in_flight += 1
        admit()                                    # overlaps the rounds in flight, if any
        if in_flight:
            try:
                finished = server.wait(stream)
            except _s.SfacError as e:
                if e.status != _s.SFAC_ETIMEOUT:
                    raise
                finished = e.finished
            in_flight -= 1
            for slot in finished:
                finish(slot)
            continue
        if not slot_req and pending:
            time.sleep(max(0.0, min(0.01, pending[0].arrival_s * time_scale - now())))
    wall = now()
    lat = np.array(list(latency.values())) if latency else np.zeros(1)
    out = {"latency": latency, "results": results, "failed": failed, "rejected": rejected, "wall_s": wall,
           "rounds": rounds,
           "point_steps": total_points, "p50_s": float(np.percentile(lat, 50)),
           "p99_s": float(np.percentile(lat, 99)), "throughput": total_points / wall if wall > 0 else 0.0}
    if evs:
        # every event has completed: each round's end was waited for
        out["gpu_busy_s"] = sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3
        out["gpu_span_s"] = evs[0][0].elapsed_time(evs[-1][1]) / 1e3
    return out
