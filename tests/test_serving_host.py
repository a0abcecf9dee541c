"""Host logic of the request loop (paper_2209_08437_gb300.serving.serve) with a
fake server: FIFO admission, back-pressure when memory is full, round
accounting and latency bookkeeping. No GPU."""
import numpy as np

import sfac_inputs as I
from paper_2209_08437_gb300 import serving
from paper_2209_08437_gb300.sfac import SFAC_ETIMEOUT, SFAC_FP32, SfacError


class FakeServer:
    """Slots with a byte budget and the round protocol of sfac_server: a round
    covers the steps of every slot that no round in flight covers yet (at most
    `chunk` each), at most two rounds are in flight, wait() completes the
    oldest and lists the slots with nothing left; a held slot makes its round
    fail like a dependency wait that gave up."""

    def __init__(self, budget, slots):
        self.prec, self.capacity = SFAC_FP32, slots
        self.budget, self.used = budget, 0
        self.active = {}                  # slot -> [steps left, bytes, field, queued, failed]
        self.admitted_order = []
        self.max_active = 0
        self.rounds = 0
        self.in_flight = []               # rounds: {slot: steps}
        self.max_in_flight = 0
        self.hold = -1

    def admit(self, problem, u0, nsteps):
        need = problem.points
        if len(self.active) >= self.capacity or self.used + need > self.budget:
            return None
        slot = min(set(range(self.capacity)) - set(self.active))
        self.active[slot] = [nsteps, need, u0.copy(), 0, False]
        self.used += need
        self.admitted_order.append(problem)
        self.max_active = max(self.max_active, len(self.active))
        return slot

    def round(self, chunk, shape=0, stream=None):
        assert len(self.in_flight) < 2
        r = {s: min(chunk, v[0] - v[3]) for s, v in self.active.items() if not v[4] and v[0] - v[3] > 0}
        if not r:
            return False
        for s, k in r.items():
            self.active[s][3] += k
        self.in_flight.append(r)
        self.rounds += 1
        self.max_in_flight = max(self.max_in_flight, len(self.in_flight))
        return True

    def wait(self, stream=None):
        if not self.in_flight:
            return []
        r = self.in_flight.pop(0)
        fail = self.hold in r
        if fail:
            self.hold = -1
        done = []
        for s, k in r.items():
            v = self.active[s]
            v[3] -= k
            if fail:
                v[4] = True
            elif not v[4]:
                v[0] -= k
                v[2] += k                 # "advance" the field
            if v[3] == 0 and (v[4] or v[0] == 0):
                done.append(s)
        if fail:
            err = SfacError(SFAC_ETIMEOUT, "wait", "held")
            err.finished = done
            raise err
        return done

    def fetch(self, slot, out=None, release=True):
        steps_left, need, field, queued, failed = self.active[slot]
        assert queued == 0
        if out is not None and not failed:
            out[...] = field
        if release:
            del self.active[slot]
            self.used -= need
        if failed:
            raise SfacError(SFAC_ETIMEOUT, "fetch", "failed")


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
        launched = super().round(chunk, shape, stream)
        if launched:
            self.log.append("round")
        return launched

    def wait(self, stream=None):
        done = super().wait(stream)
        still = sum(1 for s, v in self.active.items() if not v[4] and v[0] - v[3] > 0)  # open steps
        self.log.append(("wait", still))
        return done


def test_next_round_is_launched_before_admission():
    """After a round finishes, the loop launches the next round for the slots
    with steps that no round in flight covers before it admits queued requests
    (admission is host work that then overlaps the rounds on the GPU); requests
    admitted then join a later round."""
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


def test_two_rounds_in_flight_and_one_at_a_time():
    """The loop keeps a second round enqueued behind the running one (the
    server allows two); with max_in_flight=1 it never does. Results are the same."""
    reqs = I.serving_stream(30, rate_hz=3000.0, arrival_seed=9, sizes_2d=(32, 64), sizes_3d=(32,),
                            steps_range=(3, 20))
    outs = {}
    for m in (1, 2):
        srv = FakeServer(10 ** 9, 8)
        outs[m] = serving.serve(reqs, lambda r: np.zeros(r.problem.shape, np.float32), srv, chunk=4,
                                keep_results=True, max_in_flight=m)
        assert srv.max_in_flight == m and not srv.active and not srv.in_flight
    for r in reqs:
        assert np.all(outs[1]["results"][r.rid] == r.problem.steps)
        assert np.all(outs[2]["results"][r.rid] == r.problem.steps)


def test_failed_round_is_reported_and_the_rest_is_served():
    """A round that gives up marks its requests failed: they are reported, not
    returned, and every other request is still served to its full step count."""
    reqs = I.serving_stream(12, rate_hz=1e6, arrival_seed=4, sizes_2d=(32,), sizes_3d=(32,),
                            steps_range=(6, 10))

    class HoldFirst(FakeServer):
        def admit(self, problem, u0, nsteps):
            slot = super().admit(problem, u0, nsteps)
            if slot is not None and len(self.admitted_order) == 3:
                self.hold = slot
            return slot

    srv = HoldFirst(10 ** 9, 4)
    out = serving.serve(reqs, lambda r: np.zeros(r.problem.shape, np.float32), srv, chunk=3, keep_results=True)
    assert out["failed"], "the held round failed some requests"
    assert set(out["failed"]) | set(out["results"]) == {r.rid for r in reqs}
    assert not set(out["failed"]) & set(out["results"])
    for rid, field in out["results"].items():
        assert np.all(field == reqs[rid].problem.steps)
    assert not srv.active and srv.used == 0


def test_zero_step_requests_finish_at_admission():
    reqs = I.serving_stream(6, rate_hz=1e6, arrival_seed=2, sizes_2d=(32,), sizes_3d=(32,), steps_range=(0, 2))
    srv = FakeServer(10 ** 9, 4)
    out = serving.serve(reqs, lambda r: np.zeros(r.problem.shape, np.float32), srv, chunk=1, keep_results=True)
    assert {r.rid for r in reqs} == set(out["results"])
    assert any(r.problem.steps == 0 for r in reqs)


def test_request_larger_than_the_server_is_rejected_not_waited_for():
    """A request that does not fit even an empty server is rejected at once;
    the others are served."""
    reqs = I.serving_stream(10, rate_hz=1e6, arrival_seed=6, sizes_2d=(32, 128), sizes_3d=(32,),
                            steps_range=(2, 5))
    small = max(r.problem.points for r in reqs if r.problem.points < 128 * 128)
    srv = FakeServer(budget=small, slots=4)
    out = serving.serve(reqs, lambda r: np.zeros(r.problem.shape, np.float32), srv, chunk=2, keep_results=True)
    big = {r.rid for r in reqs if r.problem.points > small}
    assert big and set(out["rejected"]) == big
    assert set(out["results"]) == {r.rid for r in reqs} - big
