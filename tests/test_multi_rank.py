"""The benchmark's multi-GPU arithmetic (independent replicas, max-over-ranks
time) on two CPU ranks over gloo."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 * (rank + 1)                    # rank 1 is the slow one
    m = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (m, bench.replica_throughput(world, 3, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 200.0      # every rank sees the slowest time
    assert res[0][1] == pytest.approx(2 * 3 / 0.2)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_throughput(1, 4, 500.0) == pytest.approx(8.0)
