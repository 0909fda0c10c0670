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


# ---------------------------------------------------------------------------
# The rank driver (slab.run_slab_rank) with the FP64 oracle as each rank's engine
# ---------------------------------------------------------------------------

class _OracleSlab:
    """run_slab_rank's engine on the FP64 oracle: the buffer planes [b0, b1) of
    one slab, with its own pyramid; the sums are taken over its interior."""

    def __init__(self, I_m, I_s, plan, rank, nz, p):
        from paper_1204_6295_b300.slab import level_plan
        self.p = p
        self.levels = p.levels
        _, _, b0, b1 = plan[rank]
        self.pm = O.build_pyramid(I_m[b0:b1], p.levels)
        self.ps = O.build_pyramid(I_s[b0:b1], p.levels)
        self.inner = []
        for lev in range(p.levels):
            z0, z1, c0, _ = level_plan(plan, nz, lev)[rank]
            self.inner.append((z0 - c0, z1 - c0))
        self.r = {p.levels - 1: np.zeros((3,) + self.pm[-1].shape)}

    def iterate_once(self, level):
        import torch  # noqa: F401
        r = self.r[level]
        rn, dr, _, _ = O.iteration(self.pm[level], self.ps[level], r, self.p)
        a, b = self.inner[level]
        self.r[level] = rn
        return _norm_sum(dr[:, a:b]), _norm_sum(r[:, a:b])

    def level_field(self, level):
        import torch
        return torch.from_numpy(self.r[level].copy())

    def set_level_field(self, level, field):
        self.r[level] = field.numpy().astype(np.float64)

    def upsample(self, level):
        import torch
        return torch.from_numpy(O.upsample_field2(self.r[level], self.pm[level - 1].shape))


DRIVER_NZ = 32


def _driver_inputs():
    I_m = phantom.random_volume((DRIVER_NZ, NY, NX), 13, -200.0, 200.0).astype(np.float64)
    I_s = I_m + phantom.random_volume((DRIVER_NZ, NY, NX), 14, -40.0, 40.0)
    p = O.Params(patch=(3, 3, 3), sigma=0.8, levels=2, iters=[3, 3], global_shift=False)
    return I_m, I_s, p


def _driver_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1204_6295_b300.slab import halo_planes, run_slab_rank
    I_m, I_s, p = _driver_inputs()
    plan = slab_plan(DRIVER_NZ, world, halo_planes(p.patch, p.sigma, 0, 2.0, levels=2), align=2)
    eng = _OracleSlab(I_m, I_s, plan, rank, DRIVER_NZ, p)
    sums = run_slab_rank(eng, plan, rank, DRIVER_NZ, p.levels, p.iters, dist)
    z0, z1, b0, _ = plan[rank]
    out[rank] = (eng.r[0][:, z0 - b0:z1 - b0].copy(), [s.tolist() for s in sums], plan)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_rank_driver_two_levels_equals_whole_volume_oracle(world):
    """run_slab_rank on gloo ranks, each driving the FP64 oracle over its slab
    (two pyramid levels: exchanges, the allreduce, the up-sampling of each
    rank's own buffer): the assembled interiors equal the whole-volume run and
    every rank holds the whole volume's l^(k)."""
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_driver_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    I_m, I_s, p = _driver_inputs()
    ref, hist, _ = O.register(I_m, I_s, p, return_history=True)
    plan = out[0][2]
    got = np.empty_like(ref)
    for rank, (z0, z1, _, _) in enumerate(plan):
        got[:, z0:z1] = out[rank][0]
    assert np.abs(got - ref).max() <= 1e-12
    for rank in range(world):
        assert out[rank][1] == out[0][1]
    # levels in out are finest first, hist coarsest first
    for lev_sums, lev_l in zip(out[0][1][::-1], hist):
        for (sdr, sr), l in zip(lev_sums, lev_l):
            assert (sdr / sr if sr > 0 else np.inf) == pytest.approx(l, rel=1e-12)


def test_norm_stop_rule_matches_oracle():
    """disc_norm_stop_rule (the library's stop rule on summed norms, no GPU) against
    the oracle's should_stop on the same history, away from the threshold."""
    from paper_1204_6295_b300 import disc
    rng = np.random.default_rng(7)
    for trial in range(200):
        n = int(rng.integers(1, 30))
        sr = rng.uniform(1.0, 10.0, n)
        l_true = np.cumsum(rng.uniform(0.0, 0.02, n))[::-1] * rng.uniform(0.5, 2.0)
        sums = np.stack([l_true * sr, sr], 1)
        if trial % 7 == 0:
            sums[0, 1] = 0.0                           # l = inf while sum |r| = 0
        eps, window = float(rng.uniform(0.001, 0.05)), int(rng.integers(1, 12))
        l, stop = disc.norm_stop_rule(sums, window, eps)
        ref_l = [s0 / s1 if s1 > 0 else np.inf for s0, s1 in sums]
        np.testing.assert_allclose(l, np.array(ref_l, np.float32), rtol=1e-7)
        k = n - 1
        if k >= window and np.isfinite(ref_l[k - window]) and abs(ref_l[k - window] - ref_l[k] - eps) < 1e-5:
            continue                                   # float32 and float64 may decide a tie differently
        assert stop == O.should_stop(ref_l, eps, window)
    assert disc.norm_stop_rule(np.ones((12, 2)), 10, 0.0)[1] is False   # eps <= 0: fixed counts
