"""A context reused for another pair of the same size keeps its captured
iteration graphs when the scalars they hold (the fixed-point scale of I_m, the
mask thresholds) are unchanged, and rebuilds them otherwise; either way the
second pair's field equals a fresh context's bit for bit.
"""
import numpy as np
import pytest

from paper_1204_6295_b300 import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _fresh(disc, pair, **kw):
    with disc.Registration(**kw) as reg:
        reg.set_images(pair[0], pair[1])
        reg.iterate(-1)
        return reg.get_field()


@pytest.mark.parametrize("kw", [dict(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(4, 3)),
                                dict(patch=(3, 3, 3), sigma=1.0, levels=2, iters=(30, 30), stop_eps=2e-3),
                                dict(patch=(3, 3, 3), sigma=1.0, levels=1, iters=(3,), mask_mode=1)])
def test_context_reuse_matches_fresh_contexts(disc, kw):
    a = phantom.ellipsoid_pair(48, 40, 24, seed=31)
    b = phantom.ellipsoid_pair(48, 40, 24, seed=32)                   # same intensity range
    c = (2.0 * a.ct, 2.0 * a.cbct)                                    # twice the range: another scale
    pairs = [(a.ct, a.cbct), (b.ct, b.cbct), c, (a.ct, a.cbct)]
    with disc.Registration(**kw) as reg:
        for p in pairs:
            reg.set_images(np.ascontiguousarray(p[0], np.float32), np.ascontiguousarray(p[1], np.float32))
            reg.iterate(-1)
            got = reg.get_field()
            ref = _fresh(disc, (np.ascontiguousarray(p[0], np.float32), np.ascontiguousarray(p[1], np.float32)),
                         **kw)
            np.testing.assert_array_equal(got, ref)


def test_allocation_failure_is_recoverable(disc):
    """Host-side fault injection (the DISC_SW_FAULT_ALLOC test switch): disc_set_images reports
    DISC_ERR_OOM when its first device allocation fails; the failure is not sticky,
    so the same context then takes the images and registers them exactly as a
    fresh context does."""
    kw = dict(patch=(3, 3, 3), sigma=1.0, levels=2, iters=(3, 2))
    p = phantom.ellipsoid_pair(40, 32, 16, seed=33)
    ct, cbct = np.ascontiguousarray(p.ct, np.float32), np.ascontiguousarray(p.cbct, np.float32)
    with disc.Registration(**kw) as reg:
        with disc.test_switches(disc.SW_FAULT_ALLOC):
            with pytest.raises(disc.DiscError) as e:
                reg.set_images(ct, cbct)
            assert e.value.status == 4              # DISC_ERR_OOM
        reg.set_images(ct, cbct)
        reg.iterate(-1)
        got = reg.get_field()
    np.testing.assert_array_equal(got, _fresh(disc, (ct, cbct), **kw))
