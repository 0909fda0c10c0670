"""Per-kernel parity of the CUDA path against the FP64 oracle.

Each kernel is fed the same float32 inputs as the oracle (the oracle casts
them to float64).  Where a kernel's input is another kernel's output (the
correction takes the warped image, the force takes the corrected image), the
oracle is given the GPU's own float32 intermediate, so that each comparison
measures one step's arithmetic.  Bar: max |gpu - oracle| <= 1e-5 max |oracle|
per output array.
"""
import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, empty, host, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5

SHAPES_PATCHES = [
    ((13, 37, 70), (3, 3, 3)),      # ragged in x and y, several tiles
    ((11, 20, 33), (7, 5, 3)),      # anisotropic patch
    ((21, 19, 40), (11, 11, 11)),   # patch wider than the z chunk
    ((9, 33, 35), (15, 15, 15)),    # largest patch of the workloads
    ((1, 1, 1), (3, 3, 3)),         # single voxel
    ((2, 17, 1), (5, 5, 5)),        # degenerate axes
    ((6, 6, 6), (1, 1, 1)),         # 1x1x1 patch: variance 0 everywhere
    ((5, 1, 64), (3, 3, 3)),
    ((24, 52, 64), (11, 11, 11)),   # these two take the bulk-tensor-copy (TMA) form
    ((17, 33, 100), (7, 7, 7)),
]


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _half(patch):
    return tuple((p - 1) // 2 for p in patch)


def _zs_ref(Is, half, var_floor=1e-6):
    E1, E2 = O.patch_moments(Is, half)
    var = np.maximum(E2 - E1 * E1, 0.0)
    ok = var > var_floor
    return np.where(ok, (Is - E1) / np.sqrt(np.where(ok, var, 1.0)), 0.0), np.sqrt(var), ok


@pytest.mark.parametrize("shape,patch", SHAPES_PATCHES)
def test_static_norm_matches_oracle(disc, shape, patch):
    Is = ct_like(shape, 1, noise=25.0)
    qs = disc.qscale(float(np.abs(Is).max()), patch)
    zs = empty(*shape)
    disc.k_static_norm(dev(Is), zs, patch, qs)
    got = host(zs)
    ref, sd, ok = _zs_ref(Is.astype(np.float64), _half(patch))
    assert np.all(got[~ok] == 0.0)
    # compare I_s - E(S) in HU: zs times the patch STD
    err = np.abs(got - ref)[ok] * sd[ok]
    if ok.any():
        assert err.max() <= TOL * np.abs(Is).max(), err.max()


@pytest.mark.parametrize("shape,patch", SHAPES_PATCHES)
@pytest.mark.parametrize("mode", [0, 1])
def test_pass_a_matches_oracle(disc, shape, patch, mode):
    Im = ct_like(shape, 2)
    Is = ct_like(shape, 3, noise=30.0) * 0.8 + 40.0
    r = phantom.smooth_random_field(shape, 4, amp=2.5) if min(shape) > 1 else \
        phantom.random_field(shape, 4, amp=1.5)
    half = _half(patch)
    qs_s = disc.qscale(float(np.abs(Is).max()), patch)
    qs_m = disc.qscale(float(np.abs(Im).max()), patch)
    zs = empty(*shape)
    disc.k_static_norm(dev(Is), zs, patch, qs_s)
    import torch
    u, m, d = empty(3, *shape), empty(*shape), empty(*shape)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    r_d = dev(r)
    disc.k_pass_a(dev(Im), zs, r_d, u, patch, qs_m, m_out=m, d_out=d, norms_out=norms, force_mode=mode)
    m_g, d_g, u_g = host(m), host(d), host(u)
    f_g = m_g + d_g          # I'_s, formed in float64 from the GPU's m and I'_s - m
    # warp (Sec. 2.1, kernel 5)
    assert rel_err(m_g, O.warp(Im, r)) <= TOL
    # moments and correction (Eqs. 3-6) from the GPU's own warped image
    f_ref = O.correct(m_g, Is, half)
    assert rel_err(f_g, f_ref) <= TOL
    # force and update (Eq. 1, A1 steps 4-5) from the GPU's own m and I'_s
    dr_ref = O.force(m_g, f_g, mode)
    dr_g = u_g - r.astype(np.float64)
    scale = max(np.abs(dr_ref).max(), 1e-3)
    assert np.abs(dr_g - dr_ref).max() <= TOL * scale
    n_g = host(norms)
    assert n_g[0] == pytest.approx(np.sqrt((dr_ref ** 2).sum(0)).sum(), rel=1e-5, abs=1e-6)
    assert n_g[1] == pytest.approx(np.sqrt((r.astype(np.float64) ** 2).sum(0)).sum(), rel=1e-5)


def test_pass_a_affine_recovery_at_identity(disc):
    """r = 0 and I_s = alpha I_m + beta: the corrected CBCT equals I_m (App. A)."""
    shape, patch = (12, 30, 40), (5, 5, 5)
    Im = ct_like(shape, 5, noise=10.0)
    Is = (0.7 * Im.astype(np.float64) - 120.0).astype(np.float32)
    qs_s = disc.qscale(float(np.abs(Is).max()), patch)
    qs_m = disc.qscale(float(np.abs(Im).max()), patch)
    zs = empty(*shape)
    disc.k_static_norm(dev(Is), zs, patch, qs_s)
    u, m, d = empty(3, *shape), empty(*shape), empty(*shape)
    disc.k_pass_a(dev(Im), zs, dev(np.zeros((3,) + shape, np.float32)), u, patch, qs_m, m_out=m, d_out=d)
    assert np.array_equal(host(m), Im.astype(np.float64))       # identity warp is exact
    assert rel_err(host(m) + host(d), Im) <= TOL


def test_pass_a_constant_patches_give_zero_force(disc):
    """Equal images give zero force; a constant image has variance exactly 0."""
    shape, patch = (8, 20, 36), (3, 3, 3)
    Im = np.full(shape, 40.0, np.float32)
    Im[:, :, 18:] = 1000.0
    qs = disc.qscale(1000.0, patch)
    zs = empty(*shape)
    disc.k_static_norm(dev(Im), zs, patch, qs)
    interior = np.ones(shape, bool)
    interior[:, :, 16:21] = False
    assert np.all(host(zs)[interior] == 0.0)   # constant CBCT patches away from the step
    u, d = empty(3, *shape), empty(*shape)
    r0 = np.zeros((3,) + shape, np.float32)
    disc.k_pass_a(dev(Im), zs, dev(r0), u, patch, qs, d_out=d)
    assert np.all(host(d)[interior] == 0.0)       # I'_s == I_m exactly in constant patches
    assert np.all(host(u)[:, interior] == 0.0)


# the per-voxel kernel, and the z-marching one (nx >= 32, nz >= 16: ragged chunks and tiles)
@pytest.mark.parametrize("shape", [(13, 37, 70), (1, 1, 1), (4, 3, 129), (6, 1, 1), (20, 37, 70), (33, 64, 96)])
def test_warp_matches_oracle(disc, shape):
    Im = ct_like(shape, 12)
    r = phantom.random_field(shape, 13, amp=4.0)        # samples leave the volume too
    m = empty(*shape)
    disc.k_warp(dev(Im), dev(r), m)
    assert rel_err(host(m), O.warp(Im, r)) <= TOL


# nx a multiple of 4 stages the xy pass's planes as float4 vectors, other nx
# element by element; radii 1..8 cover every offset of the first tap in a vector
@pytest.mark.parametrize("shape", [(13, 37, 70), (1, 1, 1), (1, 5, 40), (40, 1, 1), (7, 16, 32), (30, 3, 65),
                                   (9, 45, 132), (6, 11, 12)])
@pytest.mark.parametrize("sigma,radius", [(1.0, 0), (1.5, 0), (2.0, 0), (0.8, 1), (1.0, 2), (1.2, 4), (2.0, 7),
                                          (2.5, 0)])
def test_gauss_matches_oracle(disc, shape, sigma, radius):
    u = phantom.random_field(shape, 6, amp=3.0)
    r = empty(3, *shape)
    disc.k_gauss(dev(u), r, sigma, radius)
    ref = O.gaussian_smooth_field(u, sigma, radius)
    assert rel_err(host(r), ref) <= TOL


@pytest.mark.parametrize("shape", [(13, 37, 70), (1, 1, 1), (5, 2, 9), (16, 16, 16)])
def test_pyramid_kernels_match_oracle(disc, shape):
    v = phantom.random_volume(shape, 7)
    nz, ny, nx = shape
    c = ((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2)
    out = empty(*c)
    disc.k_downsample2(dev(v), out)
    assert rel_err(host(out), O.downsample2(v)) <= TOL
    rc = phantom.random_field(c, 8, amp=2.0)
    rf = empty(3, *shape)
    disc.k_upsample_field2(dev(rc), rf)
    assert rel_err(host(rf), O.upsample_field2(rc, shape)) <= TOL


def test_global_shift_and_max_abs_match_oracle(disc):
    import torch
    a = phantom.random_volume((20, 33, 47), 9)
    b = phantom.random_volume((20, 33, 47), 10, -700, 300)
    out = empty(20, 33, 47)
    delta = torch.zeros(1, dtype=torch.float32, device="cuda")
    disc.k_global_shift(dev(a), dev(b), out, delta)
    ref, d = O.global_shift(a, b)
    assert float(host(delta)[0]) == pytest.approx(d, rel=1e-6)
    assert rel_err(host(out), ref) <= TOL
    mx = torch.zeros(1, dtype=torch.float32, device="cuda")
    disc.k_max_abs(dev(b), mx)
    assert float(host(mx)[0]) == float(np.abs(b).max())
