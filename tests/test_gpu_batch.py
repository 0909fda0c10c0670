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
            assert 1 <= grid <= items and zmult in (1, 2, 4, -32, -64, -(1 << 20))
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
