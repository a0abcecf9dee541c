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
    reqs = [q for q in small_stream(20) if q.problem.dim == 2][:6]
    p0 = S.make_params(reqs[0].problem.n, reqs[0].problem.alpha, reqs[0].problem.eps, reqs[0].problem.tau,
                       prec=S.SFAC_FP32)
    need = max(S.sfac_server_request_bytes(S.make_params(q.problem.n, q.problem.alpha, q.problem.eps,
                                                         q.problem.tau, prec=S.SFAC_FP32)) for q in reqs)
    assert need >= S.sfac_server_request_bytes(p0)
    with S.Server(2 * need + 4096, 8, S.SFAC_FP32) as srv:
        total = srv.info()["free_bytes"]
        a = srv.admit(reqs[0].problem, make_u0(reqs[0], np.float32), 2)
        b = srv.admit(reqs[1].problem, make_u0(reqs[1], np.float32), 2)
        assert a is not None and b is not None
        # the arena holds at most two of these requests at a time
        c = srv.admit(reqs[2].problem, make_u0(reqs[2], np.float32), 2)
        if c is None:
            srv.round(2)
            done = srv.wait()
            assert sorted(done) == sorted([a, b])
            for s in done:
                srv.fetch(s)
            c = srv.admit(reqs[2].problem, make_u0(reqs[2], np.float32), 2)
            assert c is not None
        srv.round(2)
        for s in srv.wait():
            srv.fetch(s)
        for s in (a, b, c):
            try:
                srv.fetch(s)
            except S.SfacError:
                pass
        assert srv.info()["free_bytes"] == total
        out = S.serve(reqs, lambda r: make_u0(r, np.float32), srv, chunk=4, keep_results=True)
        assert len(out["results"]) == len(reqs)
        assert srv.info()["free_bytes"] == total
