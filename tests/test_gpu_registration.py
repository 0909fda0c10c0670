"""End-to-end parity of the registration context (Algorithm A1) against the
FP64 oracle, and the behaviour of the C ABI calls on a GPU."""
import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, host

pytestmark = pytest.mark.gpu

MAX_TOL = 1e-2     # voxels, largest displacement difference after the run
MEAN_TOL = 1e-4    # voxels, mean displacement difference after the run


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _run_gpu(disc, ct, cbct, **kw):
    with disc.Registration(**kw) as reg:
        reg.set_images(ct, cbct)
        done, last = reg.iterate(-1)
        r = reg.get_field()
        hist = [reg.norm_history(l) for l in range(kw["levels"])]
        corr = reg.get_corrected()
    return r, done, last, hist, corr


def _oracle(ct, cbct, **kw):
    P = O.Params(patch=kw["patch"], sigma=kw["sigma"], radius=kw.get("radius", 0), levels=kw["levels"],
                 iters=list(kw["iters"]), force_mode=kw.get("force_mode", 0),
                 global_shift=kw.get("global_shift", True), smooth_mode=kw.get("smooth_mode", 0))
    return O.register(ct, cbct, P, return_history=True)


def _field_diff(a, b):
    d = np.sqrt(((np.asarray(a, np.float64) - b) ** 2).sum(0))
    return d.max(), d.mean()


def test_ellipsoid_phantom_single_level_matches_oracle(disc):
    """64x64x32 ellipsoid pair, patch 7^3, sigma 1, one level, 50 iterations."""
    p = phantom.ellipsoid_pair()
    kw = dict(patch=(7, 7, 7), sigma=1.0, levels=1, iters=(50,))
    r, done, last, hist, corr = _run_gpu(disc, p.ct, p.cbct, **kw)
    r_ref, hist_ref, f_ref = _oracle(p.ct, p.cbct, **kw)
    mx, mean = _field_diff(r, r_ref)
    assert mx <= MAX_TOL and mean <= MEAN_TOL, (mx, mean)
    assert done == 50
    np.testing.assert_allclose(hist[0][1:], hist_ref[0][1:], rtol=1e-3)
    assert np.isinf(hist[0][0]) and np.isinf(hist_ref[0][0])
    assert last == pytest.approx(hist_ref[0][-1], rel=1e-3)
    # corrected CBCT at the final field (Sec. 2.2): oracle on the GPU's field
    Is, _ = O.global_shift(p.ct, p.cbct)
    f_at_gpu_r = O.correct(O.warp(p.ct, r), Is, (3, 3, 3))
    assert np.abs(corr - f_at_gpu_r).max() <= 1e-5 * np.abs(f_at_gpu_r).max()


@pytest.mark.parametrize("force_mode", [0, 1])
def test_two_level_pyramid_matches_oracle(disc, force_mode):
    p = phantom.ellipsoid_pair(48, 40, 24, seed=99)
    kw = dict(patch=(5, 5, 3), sigma=1.2, levels=2, iters=(15, 15), force_mode=force_mode)
    r, done, _, _, _ = _run_gpu(disc, p.ct, p.cbct, **kw)
    r_ref, _, _ = _oracle(p.ct, p.cbct, **kw)
    mx, mean = _field_diff(r, r_ref)
    assert mx <= MAX_TOL and mean <= MEAN_TOL, (mx, mean)
    assert done == 30


def test_three_levels_odd_sizes_match_oracle(disc):
    shape = (19, 45, 51)
    ct = ct_like(shape, 11)
    u = phantom.smooth_random_field(shape, 12, amp=2.0)
    cbct = (O.warp(ct, u) * 0.9 + 30 + np.random.default_rng(13).normal(0, 10, shape)).astype(np.float32)
    kw = dict(patch=(3, 3, 3), sigma=1.0, levels=3, iters=(10, 10, 10))
    r, _, _, _, _ = _run_gpu(disc, ct, cbct, **kw)
    r_ref, _, _ = _oracle(ct, cbct, **kw)
    mx, mean = _field_diff(r, r_ref)
    assert mx <= MAX_TOL and mean <= MEAN_TOL, (mx, mean)


def test_chunked_iterate_is_bitwise_equal_and_resumable(disc):
    p = phantom.ellipsoid_pair(40, 36, 20, seed=5)
    kw = dict(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(7, 9))
    with disc.Registration(**kw) as a:
        a.set_images(p.ct, p.cbct)
        a.iterate(-1)
        ra = a.get_field()
    with disc.Registration(**kw) as b:
        b.set_images(p.ct, p.cbct)
        total = 0
        for n in (3, 1, 5, 2, 100):
            done, _ = b.iterate(n)
            total += done
        assert total == 16
        assert b.progress()[:2] == (0, 9)
        rb = b.get_field()
        np.testing.assert_array_equal(ra, rb)
    # resume from a saved coarse field
    with disc.Registration(**kw) as c:
        c.set_images(p.ct, p.cbct)
        c.iterate(7)                 # finishes the coarse level, field up-sampled
        lev, it, dims = c.progress()
        assert (lev, it) == (0, 0)
        saved = c.get_field()
    with disc.Registration(**kw) as d:
        d.set_images(p.ct, p.cbct)
        d.set_field(0, saved)
        d.iterate(-1)
        np.testing.assert_array_equal(d.get_field(), ra)


def test_device_buffers_match_host_buffers(disc):
    import torch
    p = phantom.ellipsoid_pair(32, 32, 16, seed=7)
    kw = dict(patch=(3, 3, 3), sigma=1.0, levels=1, iters=(5,))
    with disc.Registration(**kw) as a:
        a.set_images(p.ct, p.cbct)
        a.iterate(-1)
        ra = a.get_field()
    with disc.Registration(**kw) as b:
        b.set_images(dev(p.ct), dev(p.cbct))
        b.iterate(-1, sync=False)
        out = torch.empty((3, 16, 32, 32), dtype=torch.float32, device="cuda")
        b.get_field(out)
        np.testing.assert_array_equal(host(out), ra)


def test_stop_rule_ends_a_level_early(disc):
    p = phantom.ellipsoid_pair(32, 32, 16, seed=8)
    kw = dict(patch=(3, 3, 3), sigma=1.0, levels=1, iters=(400,), stop_eps=1e-2)
    with disc.Registration(**kw) as reg:
        reg.set_images(p.ct, p.cbct)
        done, last = reg.iterate(-1)
        h = reg.norm_history(0)
    assert 10 < done < 400 and len(h) == done
    assert h[-11] - h[-1] <= 1e-2
    P = O.Params(patch=(3, 3, 3), sigma=1.0, levels=1, iters=[400], stop_eps=1e-2)
    _, hist_ref, _ = O.register(p.ct, p.cbct, P, return_history=True)
    assert abs(len(hist_ref[0]) - done) <= 1


def test_errors_are_reported(disc):
    with pytest.raises(disc.DiscError):
        disc.Registration(patch=(4, 3, 3))
    with disc.Registration(patch=(3, 3, 3), levels=1, iters=(1,)) as reg:
        with pytest.raises(disc.DiscError) as e:
            reg.iterate(1)                      # no images yet
        assert e.value.status == 3
        bad = np.full((4, 4, 4), np.nan, np.float32)
        with pytest.raises(disc.DiscError) as e:
            reg.set_images(bad, bad)
        assert e.value.status == 1
        ok = np.zeros((4, 4, 4), np.float32)
        reg.set_images(ok, ok)
        reg.iterate(-1)
        assert np.all(reg.get_field() == 0.0)


@pytest.mark.parametrize("kw", [
    dict(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(15, 10), smooth_mode=1),   # Sec. 2.1 order
    dict(patch=(5, 5, 5), sigma=3.0, levels=2, iters=(10, 8)),                   # radius 9: generic Gaussian
])
def test_schedule_variants_match_oracle(disc, kw):
    p = phantom.ellipsoid_pair(48, 40, 24, seed=13)
    r, done, last, hist, _ = _run_gpu(disc, p.ct, p.cbct, **kw)
    r_ref, hist_ref, _ = _oracle(p.ct, p.cbct, **kw)
    mx, mean = _field_diff(r, r_ref)
    assert mx <= MAX_TOL and mean <= MEAN_TOL, (mx, mean)
    assert done == sum(kw["iters"])
