"""The N > 1 path of the benchmark on CPU: two gloo ranks, replicas only (walks and queries are
independent, so ranks run disjoint random streams and share nothing but the timing reduction)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [2.0, 3.5][rank]
        units = [100, 140][rank]
        out[rank] = bench.aggregate_over_ranks(seconds, units, world)
        out[10 + rank] = bench.replica_seed(2410, rank)
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    import torch.multiprocessing as mp

    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    for rank in range(2):
        t, u, v = out[rank]
        assert t == 3.5  # the slowest rank
        assert u == 240.0  # units of all ranks
        assert abs(v - 240.0 / 3.5) < 1e-12
    assert out[10] != out[11]  # disjoint walk streams


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.aggregate_over_ranks(2.0, 10, 1) == (2.0, 10, 5.0)
