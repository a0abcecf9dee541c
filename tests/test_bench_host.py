"""Host-side logic of bench.py that needs no GPU: the max-over-ranks timing
reduction of the replicas mode (world size 2, gloo) and the rate arithmetic."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [10.0 + rank, 5.0 - rank]          # rank 1 slower on the first, faster on the second
        got = bench.max_over_ranks(mine, dist, "cpu")
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == [11.0, 5.0]


def test_single_rank_identity_and_rate():
    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    # 2 ranks x 1M points x 10 steps in 5 ms of the slowest rank
    assert bench.aggregate_rate(1 << 20, 10, 2, 5.0) == pytest.approx(2 * (1 << 20) * 10 / 5e-3)


def test_flop_model():
    assert bench.pass_flops_per_point(1024) == 15 * 10 + 10
