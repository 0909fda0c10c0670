"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times: the registration context runs two iterations on the whole
volume; sampled voxels are checked against the FP64 oracle run on a crop that
contains everything those voxels depend on after two iterations (the Gaussian
radius, the patch half size, the gradient stencil and the warp displacement,
twice), with the crop's faces at the volume's faces where they coincide."""
import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like

pytestmark = pytest.mark.gpu

ITERS = 2
MAX_TOL = 1e-2
SAMPLE_TOL = 2e-3     # voxels, after two iterations on the whole volume


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _check(disc, ct, cbct, patch, sigma, samples):
    nz, ny, nx = ct.shape
    with disc.Registration(patch=patch, sigma=sigma, levels=1, iters=(ITERS,)) as reg:
        reg.set_images(ct, cbct)
        done, _ = reg.iterate(-1)
        assert done == ITERS
        r = reg.get_field()
    assert np.isfinite(r).all()
    P = O.Params(patch=patch, sigma=sigma, levels=1, iters=[ITERS])
    H, R = (patch[0] - 1) // 2, int(np.ceil(3 * sigma))
    halo = ITERS * (R + H + 2) + 2
    Is, _ = O.global_shift(ct, cbct)     # the shift cancels in the correction
    for (z, y, x) in samples:
        z0, z1 = max(0, z - halo), min(nz, z + halo + 1)
        y0, y1 = max(0, y - halo), min(ny, y + halo + 1)
        x0, x1 = max(0, x - halo), min(nx, x + halo + 1)
        sl = (slice(z0, z1), slice(y0, y1), slice(x0, x1))
        cr = np.zeros((3, z1 - z0, y1 - y0, x1 - x0))
        for _ in range(ITERS):
            cr, _, _, _ = O.iteration(ct[sl].astype(np.float64), Is[sl], cr, P)
        ref = cr[:, z - z0, y - y0, x - x0]
        got = r[:, z, y, x].astype(np.float64)
        assert np.abs(got - ref).max() <= SAMPLE_TOL, ((z, y, x), got, ref)


def test_headneck_256x256x128_patch11_sampled(disc):
    p = phantom.head_neck_pair()
    samples = [(0, 0, 0), (127, 255, 255), (64, 128, 128), (3, 100, 250), (90, 31, 32), (127, 0, 17),
               (60, 255, 140), (33, 150, 0)]
    _check(disc, p.ct, p.cbct, (11, 11, 11), 1.5, samples)


def test_large_512x512x256_patch15_sampled(disc):
    # CT-like volume with the large workload's shape and intensity range; the
    # CBCT is a shifted, scaled, noisy copy (cheaper to draw than the phantom)
    shape = (256, 512, 512)
    ct = ct_like(shape, 71)
    rng = np.random.default_rng(72)
    cbct = (np.roll(ct, (1, -2, 3), axis=(0, 1, 2)) * 0.9 + 25.0).astype(np.float32)
    cbct += rng.normal(0.0, 20.0, size=shape).astype(np.float32)
    samples = [(0, 0, 0), (255, 511, 511), (128, 256, 256), (7, 500, 33), (200, 64, 480)]
    _check(disc, ct, cbct, (15, 15, 15), 2.0, samples)
