"""Batched registration: several pairs of uneven size advanced together must give
each pair exactly the field of its own single-pair run (which the registration
tests pin to the FP64 oracle)."""
import numpy as np
import pytest

from paper_1204_6295_b300 import phantom

pytestmark = pytest.mark.gpu

DIMS = [(48, 40, 24), (32, 32, 16), (64, 48, 20), (40, 56, 30), (33, 29, 17)]
KW = dict(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(8, 8))


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


@pytest.fixture(scope="module")
def pairs():
    return [phantom.ellipsoid_pair(nx, ny, nz, seed=500 + i) for i, (nx, ny, nz) in enumerate(DIMS)]


def _single(disc, p):
    with disc.Registration(**KW) as reg:
        reg.set_images(p.ct, p.cbct)
        reg.iterate(-1)
        return reg.get_field()


def test_batched_fields_equal_single_pair_runs(disc, pairs):
    with disc.Batch(len(pairs), **KW) as b:
        for i, p in enumerate(pairs):
            b.set_images(i, p.ct, p.cbct)
        assert b.iterate(-1) == 16
        got = [b.get_field(i) for i in range(len(pairs))]
        for lev in range(2):
            items, grid, zmult = b.tuning(lev)
            assert 1 <= grid <= items and zmult in (0, 1, 2, 4, -32, -64, -(1 << 20))
        # restart and run again in two calls: identical
        b.restart()
        assert b.iterate(5) + b.iterate(-1) == 16
        again = [b.get_field(i) for i in range(len(pairs))]
    for i, p in enumerate(pairs):
        ref = _single(disc, p)
        np.testing.assert_array_equal(got[i], ref)
        np.testing.assert_array_equal(again[i], ref)


def test_batched_device_buffers_and_errors(disc, pairs):
    import torch
    with pytest.raises(disc.DiscError):
        disc.Batch(2, patch=(5, 5, 3), sigma=1.0, levels=1, iters=(1,))
    p = pairs[1]
    with disc.Batch(2, patch=(3, 3, 3), sigma=1.0, levels=1, iters=(3,)) as b:
        with pytest.raises(disc.DiscError):
            b.iterate(1)                           # images missing
        b.set_images(0, torch.from_numpy(p.ct).cuda(), torch.from_numpy(p.cbct).cuda())
        b.set_images(1, p.ct, p.cbct)
        b.iterate(-1)
        with pytest.raises(disc.DiscError) as e:
            b.set_images(0, p.ct, p.cbct)          # the schedule has started
        assert e.value.status == 3
        f0, f1 = b.get_field(0), b.get_field(1)
    np.testing.assert_array_equal(f0, f1)


# Pairs whose finest level meets the bulk-tensor-copy conditions of the batched
# moment/force kernel (nx a multiple of 4 and at least 48, ny at least 26 for
# patch 9), of uneven sizes; their coarse level takes the per-thread-load kernel.
TMA_DIMS = [(96, 64, 24), (112, 48, 20), (64, 80, 30)]
TMA_KW = dict(patch=(9, 9, 9), sigma=1.5, levels=2, iters=(4, 6))


@pytest.fixture(scope="module")
def tma_pairs():
    return [phantom.head_neck_pair(nx, ny, nz, seed=700 + i) for i, (nx, ny, nz) in enumerate(TMA_DIMS)]


@pytest.fixture(scope="module")
def tma_single(disc, tma_pairs):
    out = []
    for p in tma_pairs:
        with disc.Registration(**TMA_KW) as reg:
            reg.set_images(p.ct, p.cbct)
            reg.iterate(-1)
            out.append(reg.get_field())
    return out


# z chunking x grid: one CTA per work item, and persistent grids smaller than the
# work table, so that a CTA runs several items (of different pairs) in turn and
# carries its copy barriers' phases from one to the next
@pytest.mark.parametrize("zmult,grid", [(1, 0), (1, 5), (2, 3), (-(1 << 20), 2), (-32, 0)])
def test_batched_tma_kernel_equals_single_pair_runs(disc, tma_pairs, tma_single, zmult, grid):
    with disc.Batch(len(tma_pairs), **TMA_KW) as b:
        for i, p in enumerate(tma_pairs):
            b.set_images(i, p.ct, p.cbct)
        for lev in range(2):
            b.pin_tuning(lev, zmult, grid)
        assert b.iterate(-1) == 10
        assert b.box_path_tma(0)                   # the finest level ran k_box_tma_batch
        items, g, zm = b.tuning(0)
        assert zm == zmult and g == (items if grid == 0 else min(grid, items))
        assert grid == 0 or g < items              # persistent CTAs strode over several items
        got = [b.get_field(i) for i in range(len(tma_pairs))]
    for i in range(len(tma_pairs)):
        np.testing.assert_array_equal(got[i], tma_single[i])


@pytest.mark.parametrize("grid", [0, 7, 2])
def test_batched_wide_kernel_equals_single_pair_runs(disc, tma_pairs, tma_single, grid):
    """The wide-tile batched kernel at the finest level: one wave sharing every
    pair's (tile, plane) pairs, or a few CTAs each marching planes of several
    pairs in turn (their copy barriers' phases carried across pairs)."""
    with disc.Batch(len(tma_pairs), **TMA_KW) as b:
        for i, p in enumerate(tma_pairs):
            b.set_images(i, p.ct, p.cbct)
        b.pin_tuning(0, 0, grid)
        b.pin_tuning(1, 1, 0)
        assert b.iterate(-1) == 10
        assert b.box_path(0) == 2 and b.box_path(1) in (0, 1)
        items, g, zm = b.tuning(0)
        assert zm == 0 and (grid == 0 or g == grid)
        got = [b.get_field(i) for i in range(len(tma_pairs))]
    for i in range(len(tma_pairs)):
        np.testing.assert_array_equal(got[i], tma_single[i])


def test_batched_tuner_picks_a_tiling(disc, tma_pairs, tma_single):
    """Unpinned: the autotuner times the 32 x 16 tilings and the wide one and
    keeps the fastest; the fields are the single-pair ones whatever it picks."""
    with disc.Batch(len(tma_pairs), **TMA_KW) as b:
        for i, p in enumerate(tma_pairs):
            b.set_images(i, p.ct, p.cbct)
        b.iterate(-1)
        assert b.box_path(0) in (1, 2)            # every pair's finest level takes a bulk-copy kernel
        got = [b.get_field(i) for i in range(len(tma_pairs))]
    for i in range(len(tma_pairs)):
        np.testing.assert_array_equal(got[i], tma_single[i])


@pytest.mark.parametrize("switch,separate", [("SW_SEPARATE_WARP", 1), ("SW_FUSED_WARP", 0), (None, None)])
def test_batched_warp_placement_and_z_chunks(disc, tma_pairs, tma_single, switch, separate):
    """The Gaussian z pass and warp tuner: the warp inside the xy pass or as the
    z-marching warp kernel after the Gaussian (forced by the test switches, or chosen by
    the tuner), z chunks of any length; the fields stay the single-pair ones."""
    sw = getattr(disc, switch) if switch else 0
    with disc.test_switches(sw):
        with disc.Batch(len(tma_pairs), **TMA_KW) as b:
            for i, p in enumerate(tma_pairs):
                b.set_images(i, p.ct, p.cbct)
            assert b.iterate(-1) == 10
            for lev in range(2):
                zlen, sep = b.gauss_tuning(lev)
                assert zlen in (0, 16, 32, 64)
                assert separate is None or sep == separate
            got = [b.get_field(i) for i in range(len(tma_pairs))]
    for i in range(len(tma_pairs)):
        np.testing.assert_array_equal(got[i], tma_single[i])


def test_batched_tma_kernel_sampled_against_oracle(disc):
    """One level of two iterations, persistent grid, TMA-fed batch: sampled voxels
    of every pair against the FP64 oracle on a crop holding everything they
    depend on (as the full-size parity test does)."""
    from oracle import disc_oracle as O
    kw = dict(patch=(9, 9, 9), sigma=1.5, levels=1, iters=(2,))
    pairs = [phantom.head_neck_pair(nx, ny, nz, seed=710 + i) for i, (nx, ny, nz) in enumerate(TMA_DIMS)]
    with disc.Batch(len(pairs), **kw) as b:
        for i, p in enumerate(pairs):
            b.set_images(i, p.ct, p.cbct)
        b.pin_tuning(0, 1, 4)
        b.iterate(-1)
        assert b.box_path_tma(0)
        fields = [b.get_field(i) for i in range(len(pairs))]
    P = O.Params(patch=(9, 9, 9), sigma=1.5, levels=1, iters=[2])
    halo = 2 * (5 + 4 + 2) + 2
    for p, r in zip(pairs, fields):
        nz, ny, nx = p.ct.shape
        Is, _ = O.global_shift(p.ct, p.cbct)
        for (z, y, x) in [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, ny // 2, nx // 2), (3, ny - 5, 40)]:
            z0, z1 = max(0, z - halo), min(nz, z + halo + 1)
            y0, y1 = max(0, y - halo), min(ny, y + halo + 1)
            x0, x1 = max(0, x - halo), min(nx, x + halo + 1)
            sl = (slice(z0, z1), slice(y0, y1), slice(x0, x1))
            cr = np.zeros((3, z1 - z0, y1 - y0, x1 - x0))
            for _ in range(2):
                cr, _, _, _ = O.iteration(p.ct[sl].astype(np.float64), Is[sl], cr, P)
            ref = cr[:, z - z0, y - y0, x - x0]
            assert np.abs(r[:, z, y, x] - ref).max() <= 2e-3, ((z, y, x), r[:, z, y, x], ref)


MASK_KW = dict(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(5, 4), mask_mode=1)


def test_batched_masked_pairs_equal_single_pair_runs(disc, pairs):
    """The mask of Eqs. 7-10 in a batch: the pairs run their own schedules on
    their own streams, concurrently; each field must be its single-pair run's,
    also when the schedule is advanced in two calls."""
    sub = [pairs[0], pairs[2], pairs[4]]
    refs = []
    for p in sub:
        with disc.Registration(**MASK_KW) as reg:
            reg.set_images(p.ct, p.cbct)
            reg.iterate(-1)
            refs.append(reg.get_field())
    with disc.Batch(len(sub), **MASK_KW) as b:
        for i, p in enumerate(sub):
            b.set_images(i, p.ct, p.cbct)
        assert b.iterate(3) == 3
        assert b.iterate(-1) == 6
        got = [b.get_field(i) for i in range(len(sub))]
        with pytest.raises(disc.DiscError) as e:
            b.tuning(0)                            # no shared work table in this form
        assert e.value.status == 3
        b.restart()
        assert b.iterate(-1) == 9
        again = [b.get_field(i) for i in range(len(sub))]
    for i in range(len(sub)):
        np.testing.assert_array_equal(got[i], refs[i])
        np.testing.assert_array_equal(again[i], refs[i])


def test_batched_sec21_order_and_warp_placements(disc, tma_pairs):
    """smooth_mode 1 (r <- r + G * dr, Sec. 2.1) in a batch: the xy pass adds into r
    in place, also when the tuner times it on scratch copies; each field equals
    its single-pair run whatever the warp placement."""
    kw = dict(TMA_KW, smooth_mode=1)
    refs = []
    for p in tma_pairs:
        with disc.Registration(**kw) as reg:
            reg.set_images(p.ct, p.cbct)
            reg.iterate(-1)
            refs.append(reg.get_field())
    for sw in (disc.SW_SEPARATE_WARP, disc.SW_FUSED_WARP):
        with disc.test_switches(sw):
            with disc.Batch(len(tma_pairs), **kw) as b:
                for i, p in enumerate(tma_pairs):
                    b.set_images(i, p.ct, p.cbct)
                b.iterate(-1)
                got = [b.get_field(i) for i in range(len(tma_pairs))]
        for i in range(len(tma_pairs)):
            np.testing.assert_array_equal(got[i], refs[i])


def test_batched_patch15_sigma2_equals_single_pair_runs(disc):
    """The large workload's parameters (patch 15^3, sigma 2: R = 6) in a batch of
    uneven pairs, the shape of the bench's mixed batch: each field is its
    single-pair run's, whatever the tuner picks."""
    kw = dict(patch=(15, 15, 15), sigma=2.0, levels=2, iters=(3, 3))
    pairs = [phantom.head_neck_pair(nx, ny, nz, seed=720 + i)
             for i, (nx, ny, nz) in enumerate([(96, 64, 40), (64, 80, 32), (128, 96, 48)])]
    refs = []
    for p in pairs:
        with disc.Registration(**kw) as reg:
            reg.set_images(p.ct, p.cbct)
            reg.iterate(-1)
            refs.append(reg.get_field())
    with disc.Batch(len(pairs), **kw) as b:
        for i, p in enumerate(pairs):
            b.set_images(i, p.ct, p.cbct)
        assert b.iterate(-1) == 6
        got = [b.get_field(i) for i in range(len(pairs))]
    for i in range(len(pairs)):
        np.testing.assert_array_equal(got[i], refs[i])
