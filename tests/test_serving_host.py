"""Host logic of the request loop (paper_2209_08437_gb300.serving.serve) with a
fake server: FIFO admission, back-pressure when memory is full, round
accounting and latency bookkeeping. No GPU."""
import numpy as np

import sfac_inputs as I
from paper_2209_08437_gb300 import serving
from paper_2209_08437_gb300.sfac import SFAC_FP32


class FakeServer:
    """Slots with a byte budget; each round advances every slot by `chunk` steps."""

    def __init__(self, budget, slots):
        self.prec, self.capacity = SFAC_FP32, slots
        self.budget, self.used = budget, 0
        self.active = {}
        self.admitted_order = []
        self.max_active = 0
        self.rounds = 0

    def admit(self, problem, u0, nsteps):
        need = problem.points
        if len(self.active) >= self.capacity or self.used + need > self.budget:
            return None
        slot = min(set(range(self.capacity)) - set(self.active))
        self.active[slot] = [nsteps, need, u0.copy()]
        self.used += need
        self.admitted_order.append(problem)
        self.max_active = max(self.max_active, len(self.active))
        return slot

    def round(self, chunk, shape=0, stream=None):
        self.rounds += 1
        self._last = {s: min(chunk, v[0]) for s, v in self.active.items() if v[0] > 0}

    def wait(self, stream=None):
        done = []
        for s, k in self._last.items():
            self.active[s][0] -= k
            self.active[s][2] += k        # "advance" the field
            if self.active[s][0] == 0:
                done.append(s)
        return done

    def fetch(self, slot, out=None, release=True):
        steps_left, need, field = self.active[slot]
        if out is not None:
            out[...] = field
        if release:
            del self.active[slot]
            self.used -= need


def test_fifo_admission_backpressure_and_latency():
    reqs = I.serving_stream(30, rate_hz=5000.0, arrival_seed=3, sizes_2d=(32, 64), sizes_3d=(32,),
                            steps_range=(1, 9))
    biggest = max(r.problem.points for r in reqs)
    srv = FakeServer(budget=2 * biggest, slots=4)
    out = serving.serve(reqs, lambda r: np.zeros(r.problem.shape, np.float32), srv, chunk=3,
                        keep_results=True)
    assert set(out["latency"]) == {r.rid for r in reqs}
    assert all(v >= 0 for v in out["latency"].values())
    # admitted in arrival order, never more than memory allows
    order = sorted(reqs, key=lambda r: r.arrival_s)
    assert [p for p in srv.admitted_order] == [r.problem for r in order]
    assert srv.max_active <= 4 and srv.used == 0 and not srv.active
    # every request advanced by exactly its step count
    for r in reqs:
        assert np.all(out["results"][r.rid] == r.problem.steps)
    assert out["point_steps"] == sum(r.problem.points * r.problem.steps for r in reqs)
    assert out["p99_s"] >= out["p50_s"] >= 0


class LoggingServer(FakeServer):
    """FakeServer that records the order of its calls."""

    def __init__(self, *a):
        super().__init__(*a)
        self.log = []

    def admit(self, problem, u0, nsteps):
        slot = super().admit(problem, u0, nsteps)
        self.log.append("admit" if slot is not None else "admit-full")
        return slot

    def round(self, chunk, shape=0, stream=None):
        self.log.append("round")
        super().round(chunk, shape, stream)

    def wait(self, stream=None):
        done = super().wait(stream)
        still = sum(1 for s, v in self.active.items() if v[0] > 0)
        self.log.append(("wait", still))
        return done


def test_next_round_is_launched_before_admission():
    """After a round finishes, the loop launches the next round for the slots
    still active before it admits queued requests (admission is host work that
    then overlaps the round on the GPU); requests admitted then join the round
    after."""
    reqs = I.serving_stream(40, rate_hz=1e6, arrival_seed=5, sizes_2d=(32,), sizes_3d=(32,),
                            steps_range=(4, 12))
    srv = LoggingServer(10 ** 9, 6)
    out = serving.serve(reqs, lambda r: np.zeros(r.problem.shape, np.float32), srv, chunk=2, keep_results=True)
    assert all(np.all(out["results"][r.rid] == r.problem.steps) for r in reqs)
    log = srv.log
    checked = 0
    for i, call in enumerate(log):
        if isinstance(call, tuple) and call[1] > 0:
            # slots still had steps to do: the next call is the round, not an admission
            assert log[i + 1] == "round", log[i:i + 4]
            checked += 1
    assert checked > 0 and "admit" in log
