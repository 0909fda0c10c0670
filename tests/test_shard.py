"""Sharding of independent pairs across ranks (longest-processing-time rule).

Pinned against brute force on small instances (Graham's bound for the rule:
makespan <= (4/3 - 1/(3m)) OPT), and run on two gloo ranks on CPU: every rank
computes the same assignment of the benchmark's pair list on its own, the
shares are disjoint and cover every pair, and the slowest rank's load is
within the bound of the mean.
"""
import itertools
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1204_6295_b300 import shard


def _opt_makespan(loads, m):
    best = None
    for labels in itertools.product(range(m), repeat=len(loads)):
        t = [0] * m
        for l, r in zip(loads, labels):
            t[r] += l
        best = max(t) if best is None else min(best, max(t))
    return best


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("m", [2, 3])
def test_lpt_within_graham_bound_of_brute_force(seed, m):
    rng = np.random.default_rng(seed)
    loads = [int(v) for v in rng.integers(1, 100, size=7)]
    share = shard.lpt_assign(loads, m)
    assert sorted(i for s in share for i in s) == list(range(len(loads)))
    got = max(shard.rank_loads(loads, share))
    opt = _opt_makespan(loads, m)
    assert got <= (4.0 / 3.0 - 1.0 / (3 * m)) * opt + 1e-9


def test_lpt_edge_cases():
    assert shard.lpt_assign([], 3) == [[], [], []]
    assert shard.lpt_assign([5], 2) == [[0], []]
    assert shard.lpt_assign([3, 3, 3, 3], 2) == [[0, 2], [1, 3]]     # ties: lower index, lower rank
    with pytest.raises(ValueError):
        shard.lpt_assign([1], 0)


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
    from paper_1204_6295_b300 import phantom
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_pairs = bench.BATCH_PAIRS_PER_RANK * world
    sizes = phantom.batch_sizes(n_pairs)
    loads = [bench.schedule_units(dict(bench.BATCH_WORKLOAD, dims=d)) for d in sizes]
    share = shard.lpt_assign(loads, world)
    seen = [None] * world
    dist.all_gather_object(seen, share)          # the final gather of a sharded run
    out[rank] = (share, seen, loads)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_disjoint_complete_shares():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    share0, seen0, loads = out[0]
    share1, seen1, _ = out[1]
    assert share0 == share1 == seen0[0] == seen0[1] == seen1[0]
    mine = [set(s) for s in share0]
    assert not (mine[0] & mine[1])
    assert mine[0] | mine[1] == set(range(len(loads)))
    per_rank = shard.rank_loads(loads, share0)
    assert max(per_rank) / (sum(loads) / world) < 1.1        # 32 uneven pairs balance well
