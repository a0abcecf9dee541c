"""GPU tests of the serving layer (sfac_server_* and the request loop):
continuous batching with admission by device memory. Each result is checked
against the CPU FP64 oracle and is bit-identical alone and in the mix."""
import numpy as np
import pytest

import paper_2209_08437_gb300 as S
import sfac_inputs as I
from oracle import sfac_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_stream(count=12):
    """A compressed Poisson stream of small 2D and 3D requests."""
    return I.serving_stream(count, rate_hz=400.0, arrival_seed=11, tau=2e-3, sizes_2d=(32, 64, 128),
                            sizes_3d=(32,), steps_range=(3, 25))


def make_u0(req, dtype=np.float64):
    return np.asarray(I.request_u0(req), dtype=dtype)


@pytest.mark.parametrize("prec", [S.SFAC_FP64, S.SFAC_FP32])
def test_served_results_match_oracle(prec):
    reqs = small_stream()
    dt = np.float64 if prec == S.SFAC_FP64 else np.float32
    with S.Server(256 << 20, 16, prec) as srv:
        out = S.serve(reqs, lambda r: make_u0(r, dt), srv, chunk=7, keep_results=True)
        assert srv.info()["active"] == 0
    assert len(out["latency"]) == len(reqs)
    for r in reqs:
        ref = O.solve(r.problem, make_u0(r, dt).astype(np.float64), r.problem.steps)
        got = out["results"][r.rid].astype(np.float64)
        if prec == S.SFAC_FP64:
            assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-12, r.rid
        else:
            assert np.abs(got - ref).max() <= 1e-5, r.rid


def test_alone_equals_in_the_mix():
    reqs = small_stream()
    with S.Server(256 << 20, 16, S.SFAC_FP32) as srv:
        mixed = S.serve(reqs, lambda r: make_u0(r, np.float32), srv, chunk=5, keep_results=True)
    for r in reqs[::3]:
        with S.Server(64 << 20, 2, S.SFAC_FP32) as srv:
            alone = S.serve([r], lambda q: make_u0(q, np.float32), srv, chunk=5, keep_results=True)
        assert np.array_equal(alone["results"][r.rid], mixed["results"][r.rid]), r.rid


def test_admission_by_device_memory():
    """An arena that holds two requests of this size refuses the third
    (SFAC_ENOMEM, nothing admitted) until a result is fetched and released."""
    prob = I.Problem(n=(64, 64), alpha=(1.3, 1.6), eps=0.05, tau=2e-3)
    u0 = np.asarray(I.random_field(prob, 8, -0.9, 0.9), np.float32)
    need = S.sfac_server_request_bytes(S.make_params(prob.n, prob.alpha, prob.eps, prob.tau, prec=S.SFAC_FP32))
    with S.Server(2 * need + 4096, 8, S.SFAC_FP32) as srv:
        total = srv.info()["free_bytes"]
        a = srv.admit(prob, u0, 2)
        b = srv.admit(prob, u0, 2)
        assert a is not None and b is not None
        assert srv.admit(prob, u0, 2) is None          # no arena block left
        assert srv.info()["active"] == 2
        assert srv.round(2)
        assert sorted(srv.wait()) == sorted([a, b])
        with pytest.raises(S.SfacError) as e:
            srv.fetch(99)                               # no such slot
        assert e.value.status == S.sfac.SFAC_EINVAL
        out_a = np.empty(prob.shape, np.float32)
        srv.fetch(a, out_a)
        srv.fetch(b)
        with pytest.raises(S.SfacError) as e:
            srv.fetch(a)                                # already released
        assert e.value.status == S.sfac.SFAC_EINVAL
        c = srv.admit(prob, u0, 2)
        assert c is not None
        assert srv.round(2)
        assert srv.wait() == [c]
        out_c = np.empty(prob.shape, np.float32)
        srv.fetch(c, out_c)
        assert np.array_equal(out_a, out_c)             # the same request, alone or not
        assert srv.info()["free_bytes"] == total and srv.info()["active"] == 0
        # a stream of requests of this size and smaller: at most two in the arena at a time
        reqs = [q for q in small_stream(30) if q.problem.points <= prob.points][:6]
        out = S.serve(reqs, lambda r: make_u0(r, np.float32), srv, chunk=4, keep_results=True)
        assert len(out["results"]) == len(reqs) and not out["failed"] and not out["rejected"]
        assert srv.info()["free_bytes"] == total
        # a request larger than the whole arena is rejected, not waited for
        big = [q for q in small_stream(30) if q.problem.points > 2 * prob.points][:1]
        out = S.serve(big, lambda r: make_u0(r, np.float32), srv, chunk=4)
        assert out["rejected"] == [big[0].rid]


def test_pipelined_rounds_match_one_round_at_a_time():
    """Two rounds in flight (the second enqueued behind the first) give the
    same results, bit for bit, as one round at a time; both match the oracle."""
    reqs = small_stream(16)
    outs = {}
    for m in (1, 2):
        with S.Server(256 << 20, 16, S.SFAC_FP32) as srv:
            outs[m] = S.serve(reqs, lambda r: make_u0(r, np.float32), srv, chunk=3, keep_results=True,
                              max_in_flight=m)
    for r in reqs:
        assert np.array_equal(outs[1]["results"][r.rid], outs[2]["results"][r.rid]), r.rid
    for r in reqs[::4]:
        ref = O.solve(r.problem, make_u0(r, np.float32).astype(np.float64), r.problem.steps)
        assert np.abs(outs[2]["results"][r.rid].astype(np.float64) - ref).max() <= 1e-5, r.rid


def test_round_that_gives_up_fails_its_requests_and_the_server_recovers():
    """A held dependency wait makes one round give up: its requests are marked
    failed (their fields are partly advanced), fetching them reports
    SFAC_ETIMEOUT, and requests admitted afterwards are served and match the
    oracle."""
    reqs = [q for q in small_stream(20) if q.problem.dim == 2][:4]
    with S.Server(256 << 20, 8, S.SFAC_FP32) as srv:
        a = srv.admit(reqs[0].problem, make_u0(reqs[0], np.float32), reqs[0].problem.steps)
        b = srv.admit(reqs[1].problem, make_u0(reqs[1], np.float32), reqs[1].problem.steps)
        srv.set_wait_limit(200000, hold_slot=a)
        assert srv.round(reqs[0].problem.steps + reqs[1].problem.steps)
        with pytest.raises(S.SfacError) as e:
            srv.wait()
        assert e.value.status == S.sfac.SFAC_ETIMEOUT
        assert sorted(e.value.finished) == sorted([a, b])
        assert not srv.round(5)                          # failed slots take no further rounds
        for slot in (a, b):
            with pytest.raises(S.SfacError) as e:
                srv.fetch(slot)
            assert e.value.status == S.sfac.SFAC_ETIMEOUT
        assert srv.info()["active"] == 0
        srv.set_wait_limit(20000000)
        out = S.serve(reqs[2:], lambda r: make_u0(r, np.float32), srv, chunk=4, keep_results=True)
        assert not out["failed"]
        for r in reqs[2:]:
            ref = O.solve(r.problem, make_u0(r, np.float32).astype(np.float64), r.problem.steps)
            assert np.abs(out["results"][r.rid].astype(np.float64) - ref).max() <= 1e-5, r.rid
