"""Z-slab decomposition of one volume: the plan, the halo exchange's sources,
and the halo depth argument checked with the oracle on the CPU.

The oracle runs Algorithm A1 iterations on each slab's buffer (interior plus
halo), refreshing halo planes from their owners after every iteration, and the
interiors must equal the whole-volume run's (to FP64 rounding); a halo one
plane short of the reach of one iteration (Gaussian R + gradient 1 + patch
p_z) must not.
"""
import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom
from paper_1204_6295_b300.slab import exchange_sources, halo_planes, level_plan, slab_plan


@pytest.mark.parametrize("nz,ns,h", [(10, 1, 3), (10, 2, 3), (11, 3, 0), (64, 4, 14), (5, 5, 9), (7, 2, 100)])
def test_slab_plan_tiles_and_clips(nz, ns, h):
    plan = slab_plan(nz, ns, h)
    assert len(plan) == ns
    assert plan[0][0] == 0 and plan[-1][1] == nz
    sizes = [z1 - z0 for z0, z1, _, _ in plan]
    assert max(sizes) - min(sizes) <= 1
    for i, (z0, z1, b0, b1) in enumerate(plan):
        assert z0 < z1 and b0 == max(0, z0 - h) and b1 == min(nz, z1 + h)
        if i:
            assert plan[i - 1][1] == z0
        src = exchange_sources(plan, i)
        covered = [z for _, lo, hi in src for z in range(lo, hi)]
        assert covered == list(range(b0, b1))              # every buffer plane once, in order
        for t, lo, hi in src:
            assert plan[t][0] <= lo < hi <= plan[t][1]      # from the owner's interior


@pytest.mark.parametrize("nz,ns,h,align", [(64, 2, 22, 2), (63, 3, 8, 4), (100, 4, 16, 8), (9, 2, 4, 4)])
def test_slab_plan_aligned(nz, ns, h, align):
    plan = slab_plan(nz, ns, h, align)
    assert plan[0][0] == 0 and plan[-1][1] == nz
    for z0, z1, b0, b1 in plan:
        assert z0 % align == 0 and b0 % align == 0 and (z1 % align == 0 or z1 == nz)
        assert b0 == max(0, z0 - h) and b1 == min(nz, z1 + h)
    # at level l the cuts are the whole volume's level-l planes: halved with rounding up
    for level in range(1, align.bit_length()):
        lp = level_plan(plan, nz, level)
        nzl = nz
        for _ in range(level):
            nzl = (nzl + 1) // 2
        assert lp[0][0] == 0 and lp[-1][1] == nzl
        for (z0, z1, b0, b1), (c0, c1, d0, d1) in zip(plan, lp):
            assert c0 * (1 << level) == z0 and d0 * (1 << level) == b0
            assert d1 == (nzl if b1 == nz else b1 >> level)


def test_slab_plan_rejects():
    with pytest.raises(ValueError):
        slab_plan(3, 4, 1)
    with pytest.raises(ValueError):
        slab_plan(8, 0, 1)
    with pytest.raises(ValueError):
        slab_plan(8, 2, -1)
    with pytest.raises(ValueError):
        slab_plan(16, 2, 3, 2)                              # halo not a multiple of the alignment
    with pytest.raises(ValueError):
        slab_plan(8, 3, 4, 4)                               # fewer alignment units than slabs


def test_halo_planes():
    assert halo_planes((5, 5, 5), 1.0, 0, 6.0) == 3 + 2 + 6 + 3
    assert halo_planes((11, 11, 11), 1.5, 0, 4.0) == 5 + 5 + 4 + 3
    assert halo_planes((3, 3, 7), 2.0, 2, 0.5) == 2 + 3 + 1 + 3
    # two levels: the coarse reach counts twice in fine planes, rounded up to even
    assert halo_planes((5, 5, 5), 1.0, 0, 6.0, 2) == max(14, 2 * (3 + 2 + 3 + 3))
    assert halo_planes((3, 3, 3), 1.0, 0, 5.0, 3) == 4 * (3 + 1 + 2 + 3)


def _slab_run(I_m, I_s, r0, p, plan, iters):
    bufs = [r0[:, b0:b1].copy() for (_, _, b0, b1) in plan]
    for _ in range(iters):
        new = []
        for (z0, z1, b0, b1), rb in zip(plan, bufs):
            rn, _, _, _ = O.iteration(I_m[b0:b1], I_s[b0:b1], rb, p)
            new.append(rn)
        bufs = []
        for s, (_, _, b0, b1) in enumerate(plan):
            rb = np.empty((3, b1 - b0) + I_m.shape[1:])
            for t, lo, hi in exchange_sources(plan, s):
                tb0 = plan[t][2]
                rb[:, lo - b0:hi - b0] = new[t][:, lo - tb0:hi - tb0]
            bufs.append(rb)
    out = np.empty_like(r0)
    for rb, (z0, z1, b0, _) in zip(bufs, plan):
        out[:, z0:z1] = rb[:, z0 - b0:z1 - b0]
    return out


@pytest.mark.parametrize("force_mode,smooth_mode", [(0, 0), (1, 0), (0, 1)])
def test_slab_interiors_equal_whole_volume_oracle(force_mode, smooth_mode):
    nz, ny, nx = 30, 12, 14
    I_m = phantom.random_volume((nz, ny, nx), 3, -200.0, 200.0).astype(np.float64)
    I_s = I_m + phantom.random_volume((nz, ny, nx), 4, -40.0, 40.0)
    r0 = phantom.smooth_random_field((nz, ny, nx), 5, amp=1.5).astype(np.float64)
    p = O.Params(patch=(3, 3, 5), sigma=0.8, levels=1, iters=[3], force_mode=force_mode,
                 smooth_mode=smooth_mode)
    whole = r0
    for _ in range(3):
        whole = O.iteration(I_m, I_s, whole, p)[0]
    assert np.abs(whole[2]).max() < 2.0                    # |r_z| stays below d = 2 below
    R, pz = 3, 2
    h = halo_planes(p.patch, p.sigma, 0, 2.0)
    out = _slab_run(I_m, I_s, r0, p, slab_plan(nz, 3, h), 3)
    # the same terms per voxel; numpy may group the FP64 sums differently by extent
    assert np.abs(out - whole).max() <= 1e-12
    # one plane short of one iteration's reach on r: the interiors differ
    short = _slab_run(I_m, I_s, r0, p, slab_plan(nz, 3, R + 1 + pz - 1), 3)
    assert np.abs(short - whole).max() > 1e-6
