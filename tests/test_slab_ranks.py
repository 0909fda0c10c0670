"""The z-slab split of one volume across ranks (one slab per rank), on CPU gloo
ranks with the FP64 oracle doing each slab's iterations.

Every iteration each rank runs Algorithm A1 steps 1-6 on its buffer (interior
plus halo), adds its interior's two norm sums to the other ranks' (the scalar
allreduce of l^(k)), and refreshes its halo planes from their owners with
point-to-point messages (`slab.halo_exchange`).  The assembled interiors must
equal the whole-volume run to FP64 rounding, and the summed norms must give the
whole volume's l^(k).  Three ranks, so the middle slab exchanges with both
neighbours, and four ranks whose halo is deeper than a slab, so a buffer takes
planes from a slab that is not its neighbour.  Without the exchange the
interiors must differ.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom
from paper_1204_6295_b300.slab import allreduce_norm_sums, halo_exchange, halo_planes, slab_plan

NY, NX = 12, 14
ITERS = 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _inputs(nz):
    I_m = phantom.random_volume((nz, NY, NX), 3, -200.0, 200.0).astype(np.float64)
    I_s = I_m + phantom.random_volume((nz, NY, NX), 4, -40.0, 40.0)
    r0 = phantom.smooth_random_field((nz, NY, NX), 5, amp=1.5).astype(np.float64)
    p = O.Params(patch=(3, 3, 5), sigma=0.8, levels=1, iters=[ITERS])
    return I_m, I_s, r0, p


def _norm_sum(v):
    return float(np.sqrt((v ** 2).sum(axis=0)).sum())


def _rank_main(rank, world, port, out, nz, exchange):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    I_m, I_s, r0, p = _inputs(nz)
    plan = slab_plan(nz, world, halo_planes(p.patch, p.sigma, 0, 2.0))
    z0, z1, b0, b1 = plan[rank]
    rb = torch.from_numpy(r0[:, b0:b1].copy())
    sums = []
    for _ in range(ITERS):
        rn, dr, _, _ = O.iteration(I_m[b0:b1], I_s[b0:b1], rb.numpy(), p)
        s = torch.tensor([_norm_sum(dr[:, z0 - b0:z1 - b0]), _norm_sum(rb.numpy()[:, z0 - b0:z1 - b0])],
                         dtype=torch.float64)
        allreduce_norm_sums(s, dist)
        sums.append(s.tolist())
        rb = torch.from_numpy(np.ascontiguousarray(rn))
        if exchange:
            halo_exchange(plan, rank, rb, dist)
    out[rank] = (rb.numpy()[:, z0 - b0:z1 - b0].copy(), sums, plan)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,nz,exchange", [
    (3, 30, True),
    (3, 30, False),
    (4, 24, True),      # 6-plane slabs under a 10-plane halo: buffers span non-adjacent owners
])
def test_gloo_ranks_equal_whole_volume_oracle(world, nz, exchange):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out, nz, exchange), nprocs=world,
                       start_method="spawn")
    I_m, I_s, r0, p = _inputs(nz)
    whole, ls = r0, []
    for _ in range(ITERS):
        rn, dr, l, _ = O.iteration(I_m, I_s, whole, p)
        ls.append(l)
        whole = rn
    assert np.abs(whole[2]).max() < 2.0                    # |r_z| stays below the halo's d = 2
    plan = out[0][2]
    if world == 4:                                         # slab 0's buffer reaches slab 2
        assert plan[0][3] > plan[2][0]
    got = np.empty_like(whole)
    for rank, (z0, z1, _, _) in enumerate(plan):
        got[:, z0:z1] = out[rank][0]
    if not exchange:                                       # stale halo planes reach the interiors
        assert np.abs(got - whole).max() > 1e-6
        return
    # the same terms per voxel; numpy may group the FP64 sums differently by extent
    assert np.abs(got - whole).max() <= 1e-12
    for rank in range(world):                              # every rank holds the same summed norms
        assert out[rank][1] == out[0][1]
    for (sdr, sr), l in zip(out[0][1], ls):
        assert sdr / sr == pytest.approx(l, rel=1e-12)
