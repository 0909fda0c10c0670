"""Z-slab decomposition on the GPU: a volume registered as 2 or 3 slab contexts
with halo exchanges of r after every iteration gives the whole-volume
context's field bit for bit (same kernels, same fixed-point scales through
quant_max, same global shift), on one pyramid level and on two (slab cuts on
even planes, each slab up-sampling its own buffer at the level's end); a halo
one plane short of an iteration's reach does not.  The slabs' interior norm
sums (norm_planes) add up to the whole volume's l^(k), and the stop rule on
the summed norms ends each level at the whole-volume run's iteration.
quant_max below an image's own maximum is rejected; disc_get_level_field
returns a level's own field.
"""
import numpy as np
import pytest

from paper_1204_6295_b300 import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


@pytest.fixture(scope="module")
def pair():
    return phantom.ellipsoid_pair(48, 40, 64, seed=23)


ITERS = 8


def _whole(disc, pair, levels=1, iters=(ITERS,), **kw):
    with disc.Registration(levels=levels, iters=iters, **kw) as reg:
        reg.set_images(pair.ct, pair.cbct)
        reg.iterate(-1)
        return reg.get_field()


@pytest.mark.parametrize("nslabs,kw", [
    (2, dict(patch=(5, 5, 5), sigma=1.0)),
    (3, dict(patch=(3, 3, 7), sigma=1.5, force_mode=1)),
    (2, dict(patch=(5, 5, 3), sigma=1.0, smooth_mode=1)),
])
def test_slabs_equal_whole_volume(disc, pair, nslabs, kw):
    import torch
    from paper_1204_6295_b300.slab import SlabRegistration
    whole = _whole(disc, pair, **kw)
    assert np.abs(whole[2]).max() < 6.0
    ct, cbct = torch.from_numpy(pair.ct).cuda(), torch.from_numpy(pair.cbct).cuda()
    with SlabRegistration(nslabs, max_disp_z=6.0, iters=(ITERS,), **kw) as sr:
        sr.set_images(ct, cbct)
        assert all(b1 - b0 < 64 for _, _, b0, b1 in sr.plan)    # every slab is a proper part
        sr.iterate()
        got = sr.get_field().cpu().numpy()
    np.testing.assert_array_equal(got, whole)


@pytest.mark.parametrize("kw", [dict(patch=(5, 5, 5), sigma=1.0), dict(patch=(3, 3, 3), sigma=1.0, force_mode=1)])
def test_two_level_slabs_equal_whole_volume(disc, pair, kw):
    import torch
    from paper_1204_6295_b300.slab import SlabRegistration
    iters = (5, 4)
    whole = _whole(disc, pair, levels=2, iters=iters, **kw)
    ct, cbct = torch.from_numpy(pair.ct).cuda(), torch.from_numpy(pair.cbct).cuda()
    with SlabRegistration(2, max_disp_z=6.0, levels=2, iters=iters, **kw) as sr:
        sr.set_images(ct, cbct)
        assert all(b1 - b0 < 64 and b0 % 2 == 0 for _, _, b0, b1 in sr.plan)
        sr.iterate()
        got = sr.get_field().cpu().numpy()
    np.testing.assert_array_equal(got, whole)


def test_summed_norms_and_stop_rule(disc, pair):
    import torch
    from paper_1204_6295_b300.slab import SlabRegistration
    kw = dict(patch=(5, 5, 5), sigma=1.0)
    ct, cbct = torch.from_numpy(pair.ct).cuda(), torch.from_numpy(pair.cbct).cuda()
    # fixed counts: l^(k) of the summed interior sums against the whole volume's
    with disc.Registration(levels=2, iters=(6, 5), **kw) as reg:
        reg.set_images(pair.ct, pair.cbct)
        reg.iterate(-1)
        ref = [reg.norm_history(l) for l in range(2)]
        sums = reg.norm_sums(0)
    assert sums.shape == (5, 2) and np.all(sums > 0)
    np.testing.assert_allclose(ref[0], (sums[:, 0] / sums[:, 1]).astype(np.float32), rtol=1e-6)
    with SlabRegistration(2, max_disp_z=6.0, levels=2, iters=(6, 5), **kw) as sr:
        sr.set_images(ct, cbct)
        assert sr.iterate() == 11
        for l in range(2):
            np.testing.assert_allclose(sr.norm_history(l), ref[l], rtol=1e-5)
    # the stop rule ends the fine level early, at the same iteration in both runs
    kw2 = dict(kw, stop_eps=2e-3)
    with disc.Registration(levels=2, iters=(40, 200), **kw2) as reg:
        reg.set_images(pair.ct, pair.cbct)
        done_w, _ = reg.iterate(-1)
        whole = reg.get_field()
        hist_w = reg.norm_history(0)
    assert done_w < 240
    with SlabRegistration(2, max_disp_z=6.0, levels=2, iters=(40, 200), **kw2) as sr:
        sr.set_images(ct, cbct)
        done_s = sr.iterate()
        got = sr.get_field().cpu().numpy()
        hist_s = sr.norm_history(0)
    assert done_s == done_w and len(hist_s) == len(hist_w)
    np.testing.assert_allclose(hist_s, hist_w, rtol=1e-5)
    np.testing.assert_array_equal(got, whole)


def test_level_field(disc, pair):
    import torch
    with disc.Registration(levels=2, iters=(3, 2), patch=(3, 3, 3)) as reg:
        reg.set_images(pair.ct, pair.cbct)
        reg.iterate(3)                                   # the coarse level, then up-sampled to the fine one
        fine = reg.get_level_field(0, torch.empty((3, 64, 40, 48), device="cuda"))
        np.testing.assert_array_equal(fine.cpu().numpy(), reg.get_field())
        coarse = reg.get_level_field(1, np.empty((3, 32, 20, 24), np.float32))
        up = torch.empty((3, 64, 40, 48), device="cuda")
        disc.k_upsample_field2(torch.from_numpy(coarse).cuda(), up)
        np.testing.assert_array_equal(up.cpu().numpy(), fine.cpu().numpy())
        with pytest.raises(disc.DiscError):
            reg.get_level_field(2, np.empty((3, 16, 10, 12), np.float32))


def test_short_halo_differs(disc, pair):
    import torch
    from paper_1204_6295_b300.slab import SlabRegistration
    kw = dict(patch=(5, 5, 5), sigma=1.0)
    whole = _whole(disc, pair, **kw)
    ct, cbct = torch.from_numpy(pair.ct).cuda(), torch.from_numpy(pair.cbct).cuda()
    with SlabRegistration(2, halo=3 + 1 + 2 - 1, iters=(ITERS,), **kw) as sr:
        sr.set_images(ct, cbct)
        sr.iterate()
        got = sr.get_field().cpu().numpy()
    assert np.abs(got - whole).max() > 1e-4


def test_quant_max_bounds(disc, pair):
    mx = float(np.abs(pair.ct).max())
    with disc.Registration(levels=1, iters=(2,), patch=(3, 3, 3), global_shift=False,
                           quant_max=(0.5 * mx, 0.0)) as reg:
        with pytest.raises(disc.DiscError):
            reg.set_images(pair.ct, pair.cbct)
    # a bound equal to the maximum gives the default scales: the same field
    fields = []
    for q in ((0.0, 0.0), (mx, float(np.abs(pair.cbct).max()))):
        with disc.Registration(levels=1, iters=(3,), patch=(3, 3, 3), global_shift=False, quant_max=q) as reg:
            reg.set_images(pair.ct, pair.cbct)
            reg.iterate(-1)
            fields.append(reg.get_field())
    np.testing.assert_array_equal(fields[0], fields[1])
