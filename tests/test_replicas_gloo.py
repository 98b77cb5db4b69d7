"""N > 1 path of the bench: independent replicas, whole-job totals over ranks.

Two CPU ranks over gloo (127.0.0.1) call the same aggregation the bench uses
under torchrun with NCCL: DoF-applies are summed, times are the maximum over
ranks, so the reported throughput is all ranks' work over the slowest rank's
time.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r did (r + 1) * 1e6 DoF-applies in 10 (r + 1) ms of J.w, region 2 (r + 1) s
        res = bench.aggregate_replicas(1e6 * (rank + 1), 10.0 * (rank + 1), 2.0 * (rank + 1), world, "cpu")
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        applies, jv_ms, t_region = res[rank]
        assert applies == pytest.approx(3e6)   # summed: 1e6 + 2e6
        assert jv_ms == pytest.approx(20.0)     # slowest rank
        assert t_region == pytest.approx(4.0)
    # the bench's value: all ranks' DoF-applies over the slowest rank's J.w time
    value = res[0][0] / (res[0][1] / 1e3) / 1e9
    assert value == pytest.approx(0.15)


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_replicas(5.0, 2.0, 1.0, 1, "cpu") == (5.0, 2.0, 1.0)
