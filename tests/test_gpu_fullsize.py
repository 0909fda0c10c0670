"""Parity at the workloads' full sizes and with their own schedules.

1. Full volumes, in the launch configuration the benchmark times. The registration
   context runs two iterations on the whole volume (the wide-tile iteration pass,
   the Gaussian z pass and the xy pass with the fused warp: the finest level's kernels).
   Sampled voxels are checked against the FP64 oracle run on a crop that contains
   everything those voxels depend on after two iterations: the Gaussian radius, the
   patch half size, the gradient stencil and the warp displacement, twice. Where they
   coincide, the crop's faces are the volume's faces. The samples are every corner,
   the centre, and seeded interior and face voxels. The bars are the end-to-end ones,
   taken over the samples: 1e-2 voxel max and 1e-4 voxel mean.
2. Multi-level schedules at the workloads' parameters. The head-and-neck schedule
   (patch 11³, σ 1.5, three levels) and the large pair's four-level pyramid (patch
   15³, σ 2, four levels) run on smaller pairs from the same generator, whole. The
   field is compared with the oracle's registration everywhere, at the same bars.
"""
import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like

pytestmark = pytest.mark.gpu

ITERS = 2
MAX_TOL = 1e-2       # voxels
MEAN_TOL = 1e-4      # voxels


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _samples(shape, seed, n_interior=12, n_face=6):
    nz, ny, nx = shape
    out = [(z, y, x) for z in (0, nz - 1) for y in (0, ny - 1) for x in (0, nx - 1)]
    out.append((nz // 2, ny // 2, nx // 2))
    rng = np.random.default_rng(seed)
    for _ in range(n_interior):
        out.append((int(rng.integers(0, nz)), int(rng.integers(0, ny)), int(rng.integers(0, nx))))
    for k in range(n_face):                       # a voxel on each of the six faces
        p = [int(rng.integers(0, nz)), int(rng.integers(0, ny)), int(rng.integers(0, nx))]
        ax = k // 2
        p[ax] = 0 if k % 2 == 0 else shape[ax] - 1
        out.append(tuple(p))
    return out


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
    diffs = []
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
        diffs.append(float(np.sqrt(((got - ref) ** 2).sum())))
    diffs = np.array(diffs)
    worst = samples[int(diffs.argmax())]
    assert diffs.max() <= MAX_TOL and diffs.mean() <= MEAN_TOL, (diffs.max(), diffs.mean(), worst)


def test_headneck_256x256x128_patch11_sampled(disc):
    p = phantom.head_neck_pair()
    samples = _samples(p.ct.shape, 5) + [(3, 100, 250), (90, 31, 32), (127, 0, 17), (60, 255, 140), (33, 150, 0)]
    _check(disc, p.ct, p.cbct, (11, 11, 11), 1.5, samples)


def test_large_512x512x256_patch15_sampled(disc):
    # CT-like volume with the large workload's shape and intensity range; the
    # CBCT is a shifted, scaled, noisy copy (cheaper to draw than the phantom)
    shape = (256, 512, 512)
    ct = ct_like(shape, 71)
    rng = np.random.default_rng(72)
    cbct = (np.roll(ct, (1, -2, 3), axis=(0, 1, 2)) * 0.9 + 25.0).astype(np.float32)
    cbct += rng.normal(0.0, 20.0, size=shape).astype(np.float32)
    samples = _samples(shape, 6) + [(7, 500, 33), (200, 64, 480)]
    _check(disc, ct, cbct, (15, 15, 15), 2.0, samples)


@pytest.mark.parametrize("dims,kw", [
    # the head-and-neck schedule's parameters (patch 11^3, sigma 1.5, three levels)
    ((96, 96, 48), dict(patch=(11, 11, 11), sigma=1.5, levels=3, iters=(8, 8, 6))),
    # the large pair's four-level pyramid (patch 15^3, sigma 2, four levels)
    ((128, 128, 64), dict(patch=(15, 15, 15), sigma=2.0, levels=4, iters=(5, 5, 4, 3))),
])
def test_workload_schedules_match_oracle(disc, dims, kw):
    p = phantom.head_neck_pair(*dims, seed=91)
    with disc.Registration(**kw) as reg:
        reg.set_images(p.ct, p.cbct)
        done, _ = reg.iterate(-1)
        r = reg.get_field()
    assert done == sum(kw["iters"])
    P = O.Params(patch=kw["patch"], sigma=kw["sigma"], levels=kw["levels"], iters=list(kw["iters"]))
    ref = O.register(p.ct, p.cbct, P)
    d = np.sqrt(((r.astype(np.float64) - ref) ** 2).sum(0))
    assert d.max() <= MAX_TOL and d.mean() <= MEAN_TOL, (d.max(), d.mean())
