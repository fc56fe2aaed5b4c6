"""Replica timing of bench.py across ranks (world size 2, gloo on CPU): every
rank sees the slowest rank's time and the whole-job rate counts all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 + 7.5 * rank             # rank 1 is the slow one
        worst = bench.max_over_ranks(ms, device="cpu")
        rate = bench.aggregate_rate(1000.0, 4, world, worst)
        out[rank] = (worst, rate)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 17.5
    assert res[0][1] == res[1][1] == pytest.approx(1000.0 * 4 * 2 / 0.0175)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, device="cpu") == 3.25
    assert bench.aggregate_rate(10.0, 2, 1, 1000.0) == 20.0
