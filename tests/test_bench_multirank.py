"""The N > 1 benchmark path: every rank plans its own replica and rank 0
reports the slowest rank's step time and the sum of the ranks' work.  Two
gloo ranks on the CPU (no GPU, no NCCL)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ms, units, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.aggregate(ms[rank], units[rank], world, dist, device="cpu")
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank_and_sums_work():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    ms = [0.07, 0.09]
    units = [8464384.0, 8464384.0]
    port = _free_port()
    mp.spawn(_worker, args=(2, port, ms, units, out), nprocs=2, join=True)
    for r in range(2):
        t, u = out[r]
        assert t == pytest.approx(0.09)
        assert u == pytest.approx(2 * 8464384.0)


def test_single_rank_aggregation_is_the_identity():
    import bench
    assert bench.aggregate(0.05, 123.0, 1) == (0.05, 123.0)
