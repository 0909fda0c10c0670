"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks with different
step times agree on the slowest one, and the whole-job throughput counts every
rank's work (weak scaling, replicas of the same workload)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.reduce_max(dist, 1.0 + rank, device="cpu")
    out[rank] = (t, bench.job_throughput(10 ** 9, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == pytest.approx(world * 1.0 / 2.0)


def test_units_and_levels():
    import bench
    w = bench.WORKLOADS["headneck-256x256x128"]
    assert bench.schedule_units(w) == 956825600
    assert bench.level_dims((5, 3, 1), 3) == [(5, 3, 1), (3, 2, 1), (2, 1, 1)]
