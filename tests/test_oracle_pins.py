"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each test checks it against
brute force written independently (scalar loops, different formulation), a
closed form, a hand-worked example under ``tests/golden/``, a library routine
that coincides with the definition in a special case, or an invariant.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------- warp (Sec. 2.1)

def _trilinear_scalar(img, px, py, pz):
    """Scalar trilinear as nested lerps (x, then y, then z) with clamping."""
    nz, ny, nx = img.shape
    px = min(max(px, 0.0), nx - 1)
    py = min(max(py, 0.0), ny - 1)
    pz = min(max(pz, 0.0), nz - 1)
    x0, y0, z0 = int(math.floor(px)), int(math.floor(py)), int(math.floor(pz))
    x1, y1, z1 = min(x0 + 1, nx - 1), min(y0 + 1, ny - 1), min(z0 + 1, nz - 1)
    tx, ty, tz = px - x0, py - y0, pz - z0

    def lx(z, y):
        return img[z, y, x0] + tx * (img[z, y, x1] - img[z, y, x0])

    def ly(z):
        return lx(z, y0) + ty * (lx(z, y1) - lx(z, y0))

    return ly(z0) + tz * (ly(z1) - ly(z0))


def test_warp_identity_is_exact():
    img = phantom.random_volume((5, 6, 7), 1)
    assert np.array_equal(O.warp(img, np.zeros((3, 5, 6, 7))), img.astype(np.float64))


def test_warp_integer_shift_is_index_shift():
    img = phantom.random_volume((6, 7, 8), 2).astype(np.float64)
    r = np.zeros((3, 6, 7, 8))
    r[0], r[2] = 1.0, -2.0
    z, y, x = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    ref = img[np.clip(z - 2, 0, 5), y, np.clip(x + 1, 0, 7)]
    assert np.array_equal(O.warp(img, r), ref)


def test_warp_reproduces_affine_images():
    # trilinear interpolation reproduces an affine function exactly
    nz, ny, nx = 6, 7, 8
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    img = 2.0 * x - 3.0 * y + 0.5 * z + 7.0
    rng = _rng(3)
    r = rng.uniform(-0.9, 0.9, size=(3, nz, ny, nx))
    px = np.clip(x + r[0], 0, nx - 1)
    py = np.clip(y + r[1], 0, ny - 1)
    pz = np.clip(z + r[2], 0, nz - 1)
    ref = 2.0 * px - 3.0 * py + 0.5 * pz + 7.0
    np.testing.assert_allclose(O.warp(img, r), ref, rtol=0, atol=1e-12)


def test_warp_matches_scalar_bruteforce():
    img = phantom.random_volume((4, 5, 6), 4).astype(np.float64)
    r = phantom.random_field((4, 5, 6), 5, amp=3.0).astype(np.float64)  # leaves the grid
    out = O.warp(img, r)
    for z in range(4):
        for y in range(5):
            for x in range(6):
                ref = _trilinear_scalar(img, x + r[0, z, y, x], y + r[1, z, y, x], z + r[2, z, y, x])
                assert abs(out[z, y, x] - ref) <= 1e-10 * (1 + abs(ref))


def test_warp_region_equals_warp_on_the_full_grid():
    img = phantom.random_volume((7, 8, 9), 27).astype(np.float64)
    r = phantom.random_field((7, 8, 9), 28, amp=4.0).astype(np.float64)
    full = O.warp(img, r)
    sub = O.warp_region(img, r[:, 2:6, 1:7, 3:9], (3, 1, 2))
    np.testing.assert_array_equal(sub, full[2:6, 1:7, 3:9])


# ------------------------------------------------------------ moments (Eq. 3)

def _patch(X, z, y, x, half):
    hx, hy, hz = half
    nz, ny, nx = X.shape
    vals = []
    for zz in range(max(0, z - hz), min(nz, z + hz + 1)):
        for yy in range(max(0, y - hy), min(ny, y + hy + 1)):
            for xx in range(max(0, x - hx), min(nx, x + hx + 1)):
                vals.append(X[zz, yy, xx])
    return np.array(vals)


@pytest.mark.parametrize("half", [(1, 1, 1), (1, 2, 1), (2, 1, 0), (3, 3, 2)])
def test_patch_moments_match_bruteforce(half):
    X = phantom.random_volume((5, 6, 7), 6).astype(np.float64)
    E1, E2 = O.patch_moments(X, half)
    n = O.box_count(X.shape, half)
    for z in range(5):
        for y in range(6):
            for x in range(7):
                v = _patch(X, z, y, x, half)
                assert n[z, y, x] == v.size
                assert abs(E1[z, y, x] - v.mean()) <= 1e-9
                assert abs(E2[z, y, x] - (v * v).mean()) <= 1e-6


def test_constant_image_has_zero_patch_variance():
    X = np.full((5, 6, 7), 37.25)
    E1, E2 = O.patch_moments(X, (2, 2, 2))
    assert np.all(O.patch_std(E1, E2) <= 1e-6)
    assert np.allclose(E1, 37.25, rtol=0, atol=1e-12)


# -------------------------------------------------- moment matching (Eqs. 2-6)

def test_golden_moment_matching_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "moment_matching_1d.json")))
    M = np.array(g["M"]).reshape(1, 1, 3)
    S = np.array(g["S"]).reshape(1, 1, 3)
    half = tuple((p - 1) // 2 for p in g["patch"])
    a, b = O.intensity_coefficients(M, S, half)
    np.testing.assert_allclose(a.ravel(), g["a"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b.ravel(), g["b"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.correct(M, S, half).ravel(), g["corrected"], rtol=1e-12)


def test_corrected_patch_moments_equal_moving_patch_moments():
    # Eq. (4): with a(x), b(x) from Eqs. (5)-(6), the transformed patch a S + b
    # has the same first and second moments as the moving patch M.
    m = phantom.random_volume((4, 5, 6), 7, -300, 900).astype(np.float64)
    s = phantom.random_volume((4, 5, 6), 8, -800, 200).astype(np.float64)
    half = (1, 2, 1)
    a, b = O.intensity_coefficients(m, s, half)
    for z in range(4):
        for y in range(5):
            for x in range(6):
                M = _patch(m, z, y, x, half)
                Sp = a[z, y, x] * _patch(s, z, y, x, half) + b[z, y, x]
                assert abs(Sp.mean() - M.mean()) <= 1e-9 * (1 + abs(M.mean()))
                assert abs((Sp ** 2).mean() - (M ** 2).mean()) <= 1e-9 * (M ** 2).mean()


def test_affine_intensity_map_is_recovered_exactly():
    # I_s = alpha I_m + beta with alpha > 0 gives a = 1/alpha, b = -beta/alpha
    # in every patch (Appendix A.5-A.7), so I'_s == I_m at every voxel.
    m = phantom.random_volume((6, 7, 8), 9).astype(np.float64)
    s = 0.62 * m - 137.0
    out = O.correct(m, s, (2, 1, 1))
    np.testing.assert_allclose(out, m, rtol=0, atol=1e-9 * np.abs(m).max())


def test_constant_static_patch_gives_moving_mean():
    m = phantom.random_volume((5, 5, 5), 10).astype(np.float64)
    s = np.full((5, 5, 5), 12.0)
    E1, _ = O.patch_moments(m, (1, 1, 1))
    np.testing.assert_allclose(O.correct(m, s, (1, 1, 1)), E1, rtol=0, atol=1e-9)


# -------------------------------------------------------- gradient (kernel 3)

def test_gradient_matches_numpy_gradient():
    f = phantom.random_volume((5, 6, 7), 11).astype(np.float64)
    g = O.gradient(f)
    gz, gy, gx = np.gradient(f, edge_order=1)
    np.testing.assert_allclose(g[0], gx, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g[1], gy, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g[2], gz, rtol=0, atol=1e-12)


# ----------------------------------------------------------- force (Eq. 1)

def test_golden_thirion_force_worked_examples():
    g = json.load(open(os.path.join(GOLDEN, "thirion_force_1d.json")))
    for case in g["cases"]:
        f = np.array(case["f"]).reshape(1, 1, 3)
        m = np.array(case["m"]).reshape(1, 1, 3)
        dr = O.force(m, f, O.FORCE_THIRION)
        np.testing.assert_allclose(dr[0].ravel(), case["dr_x"], rtol=1e-12, atol=1e-15)
        assert np.all(dr[1] == 0) and np.all(dr[2] == 0)


@pytest.mark.parametrize("mode", [O.FORCE_THIRION, O.FORCE_DOUBLE])
def test_equal_images_give_zero_force(mode):
    f = phantom.random_volume((5, 6, 7), 12).astype(np.float64)
    assert np.all(O.force(f, f, mode) == 0.0)


def test_thirion_force_bounded_by_half_and_parallel_to_gradient():
    m = phantom.random_volume((6, 7, 8), 13).astype(np.float64)
    f = phantom.random_volume((6, 7, 8), 14).astype(np.float64)
    dr = O.force(m, f, O.FORCE_THIRION)
    assert np.sqrt((dr ** 2).sum(0)).max() <= 0.5 + 1e-12
    g = O.gradient(f)
    cross = np.cross(np.moveaxis(dr, 0, -1), np.moveaxis(g, 0, -1))
    assert np.abs(cross).max() <= 1e-9 * np.abs(g).max()


def test_double_force_is_sum_of_two_passive_terms():
    # Eq. (1): the double force adds the same expression with grad I_m^(k)
    m = phantom.random_volume((5, 6, 7), 15).astype(np.float64)
    f = phantom.random_volume((5, 6, 7), 16).astype(np.float64)
    d2 = O.force(m, f, O.FORCE_DOUBLE)
    # swapping roles of the gradient image: term 2 is the Thirion force with grad m
    gm = np.stack(np.gradient(m, edge_order=1)[::-1])
    diff = f - m
    term2 = diff * gm / ((gm ** 2).sum(0) + diff ** 2)
    np.testing.assert_allclose(d2 - O.force(m, f, O.FORCE_THIRION), term2, rtol=1e-10, atol=1e-13)
    assert np.sqrt((d2 ** 2).sum(0)).max() <= 1.0 + 1e-12


# ------------------------------------------------------ Gaussian (A1 step 6)

def test_gaussian_matches_bruteforce_3d():
    v = phantom.random_volume((5, 6, 7), 17).astype(np.float64)
    sigma, R = 1.1, 2
    w = np.exp(-np.arange(-R, R + 1) ** 2 / (2 * sigma ** 2))
    out = O.gaussian_smooth(v, sigma, R)
    nz, ny, nx = v.shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                num = den = 0.0
                for dz in range(-R, R + 1):
                    for dy in range(-R, R + 1):
                        for dx in range(-R, R + 1):
                            zz, yy, xx = z + dz, y + dy, x + dx
                            if 0 <= zz < nz and 0 <= yy < ny and 0 <= xx < nx:
                                wt = w[dz + R] * w[dy + R] * w[dx + R]
                                num += wt * v[zz, yy, xx]
                                den += wt
                assert abs(out[z, y, x] - num / den) <= 1e-9


def test_gaussian_interior_matches_scipy():
    from scipy.ndimage import gaussian_filter
    v = phantom.random_volume((20, 21, 22), 18).astype(np.float64)
    sigma = 1.5
    R = int(math.ceil(3 * sigma))
    ours = O.gaussian_smooth(v, sigma)
    ref = gaussian_filter(v, sigma, truncate=R / sigma, mode="constant")
    sl = (slice(R, -R),) * 3
    np.testing.assert_allclose(ours[sl], ref[sl], rtol=0, atol=1e-9)


def test_gaussian_preserves_constants_and_taps_formula():
    v = np.full((4, 5, 6), -3.5)
    np.testing.assert_allclose(O.gaussian_smooth(v, 2.0), v, rtol=0, atol=1e-12)
    w = O.gaussian_taps(1.0)
    assert len(w) == 7 and w[3] == 1.0
    np.testing.assert_allclose(w[0], math.exp(-4.5), rtol=1e-15)


# -------------------------------------------------------- pyramid (Sec. 2.3)

def test_downsample_bruteforce_and_constants():
    v = phantom.random_volume((5, 6, 7), 19).astype(np.float64)
    d = O.downsample2(v)
    assert d.shape == (3, 3, 4)
    for z in range(3):
        for y in range(3):
            for x in range(4):
                cell = v[2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * x:2 * x + 2]
                assert abs(d[z, y, x] - cell.mean()) <= 1e-12
    np.testing.assert_allclose(O.downsample2(np.full((5, 6, 7), 4.0)), 4.0, rtol=0, atol=1e-12)


def test_upsample_constant_and_linear_fields():
    c = np.full((3, 3, 4, 5), 1.25)
    up = O.upsample_field2(c, (6, 8, 9))
    np.testing.assert_allclose(up, 2.5, rtol=0, atol=1e-12)
    # a field equal to the coarse x index maps to 2 * (i - 0.5) / 2 = i - 0.5 inside
    lin = np.zeros((3, 4, 4, 6))
    lin[0] = np.arange(6)[None, None, :]
    up = O.upsample_field2(lin, (8, 8, 12))
    np.testing.assert_allclose(up[0][:, :, 1:11],
                               np.broadcast_to(np.arange(1, 11) - 0.5, (8, 8, 10)), atol=1e-12)


def test_level_dims():
    assert O.level_dims((256, 256, 128), 3) == [(256, 256, 128), (128, 128, 64), (64, 64, 32)]
    assert O.level_dims((5, 3, 1), 3) == [(5, 3, 1), (3, 2, 1), (2, 1, 1)]


# ----------------------------------------------- norm and shift (Sec. 2.3)

def test_relative_norm_hand_example():
    dr = np.zeros((3, 1, 1, 2))
    r = np.zeros((3, 1, 1, 2))
    dr[0, 0, 0, 0], dr[1, 0, 0, 0] = 3.0, 4.0      # |dr| = 5
    dr[2, 0, 0, 1] = 1.0                            # |dr| = 1
    r[0, 0, 0, 1] = 2.0                             # |r| = 2
    assert O.relative_norm(dr, r) == pytest.approx(3.0)
    assert O.relative_norm(dr, np.zeros_like(r)) == math.inf
    h = [math.inf, 0.5] + [0.4] * 9
    assert not O.should_stop(h[:-1], 1e-4)
    assert O.should_stop(h + [0.49995], 1e-4)
    assert not O.should_stop(h + [0.3], 1e-4)


def test_global_shift_equalises_means():
    a = phantom.random_volume((4, 5, 6), 20).astype(np.float64)
    b = phantom.random_volume((4, 5, 6), 21, -500, 100).astype(np.float64)
    s, d = O.global_shift(a, b)
    assert abs(s.mean() - a.mean()) <= 1e-9
    assert d == pytest.approx(a.mean() - b.mean())


# ------------------------------------------- whole loop (Algorithm A1, Sec. 3.1)

def test_phantom_deformation_is_recovered():
    """The known smooth deformation of the ellipsoid phantom is recovered.

    Sec. 3.1: DISC registers the CT to an artifact-laden CBCT.  After 50
    iterations the warped CT is far closer to the artifact-free CBCT and the
    field error on edges (where the deformation is observable) drops; flipping
    the force sign (the rejected reading of Eq. 1) makes both worse.
    """
    p = phantom.ellipsoid_pair()
    u = p.u_true.astype(np.float64)
    band = np.sqrt((O.gradient(p.cbct_primary) ** 2).sum(0)) > 20
    P = O.Params(patch=(7, 7, 7), sigma=1.0, levels=1, iters=[50])
    r = O.register(p.ct, p.cbct, P)

    def err(f):
        return np.sqrt(((f - u) ** 2).sum(0))[band].mean()

    def dissim(f):
        return np.sqrt(((O.warp(p.ct, f) - p.cbct_primary) ** 2).mean())

    z = np.zeros_like(u)
    assert dissim(r) < 0.5 * dissim(z)
    assert err(r) < 0.9 * err(z)
    # plain demons on the same cupped CBCT (no correction) does no better
    Is, _ = O.global_shift(p.ct, p.cbct)
    rd = np.zeros_like(u)
    for _ in range(50):
        rd = O.gaussian_smooth_field(rd + O.force(O.warp(p.ct, rd), Is), 1.0)
    assert err(r) <= err(rd) + 1e-9
    # the opposite sign moves away from the solution
    rf = np.zeros_like(u)
    for _ in range(10):
        m = O.warp(p.ct, rf)
        rf = O.gaussian_smooth_field(rf - O.force(m, O.correct(m, Is, P.half)), 1.0)
    assert dissim(rf) > dissim(z)


# ------------------------------------------- differentiable form (SSD adjoint)

def _smooth_pair(shape, seed):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rng = _rng(seed)
    img = np.zeros(shape)
    for _ in range(4):
        k = rng.uniform(0.2, 0.7, size=3)
        img += 300 * np.sin(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, 6))
    s = 0.7 * img + 40 * np.sin(0.3 * x) + rng.normal(0, 5, size=shape)
    return img, s


def test_ssd_adjoint_matches_central_differences():
    shape = (6, 7, 8)
    I_m, I_s = _smooth_pair(shape, 22)
    r = phantom.smooth_random_field(shape, 23, amp=1.2).astype(np.float64)
    half = (1, 1, 1)
    g = O.ssd_grad(I_m, I_s, r, half)
    eps = 1e-4
    rng = _rng(24)
    nz, ny, nx = shape
    checked = 0
    for _ in range(40):
        c, z, y, x = rng.integers(0, 3), rng.integers(1, nz - 1), rng.integers(1, ny - 1), rng.integers(1, nx - 1)
        pos = (x, y, z)[c] + r[c, z, y, x]
        frac = pos - math.floor(pos)
        if frac < 10 * eps or frac > 1 - 10 * eps:
            continue
        rp = r.copy(); rp[c, z, y, x] += eps
        rm = r.copy(); rm[c, z, y, x] -= eps
        fd = (O.ssd_loss(I_m, I_s, rp, half) - O.ssd_loss(I_m, I_s, rm, half)) / (2 * eps)
        assert abs(fd - g[c, z, y, x]) <= 1e-5 * max(1.0, abs(fd)), (c, z, y, x, fd, g[c, z, y, x])
        checked += 1
    assert checked >= 20


def test_ssd_adjoint_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    shape = (5, 6, 7)
    I_m, I_s = _smooth_pair(shape, 25)
    r = phantom.smooth_random_field(shape, 26, amp=1.5).astype(np.float64)
    half = (1, 1, 1)
    g = O.ssd_grad(I_m, I_s, r, half)

    # independent forward written with torch ops (gather-based trilinear,
    # conv3d box means), differentiated by autograd in float64
    Im = torch.tensor(I_m)
    Is = torch.tensor(I_s)
    rt = torch.tensor(r, requires_grad=True)
    nz, ny, nx = shape
    zz, yy, xx = torch.meshgrid(torch.arange(nz, dtype=torch.float64),
                                torch.arange(ny, dtype=torch.float64),
                                torch.arange(nx, dtype=torch.float64), indexing="ij")
    p = [torch.clamp(xx + rt[0], 0, nx - 1), torch.clamp(yy + rt[1], 0, ny - 1),
         torch.clamp(zz + rt[2], 0, nz - 1)]
    i0 = [torch.floor(q).detach().long() for q in p]
    t = [q - i.double() for q, i in zip(p, i0)]
    i1 = [torch.clamp(i + 1, max=n - 1) for i, n in zip(i0, (nx, ny, nz))]
    m = 0
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                w = (t[0] if cx else 1 - t[0]) * (t[1] if cy else 1 - t[1]) * (t[2] if cz else 1 - t[2])
                m = m + w * Im[(i1 if cz else i0)[2], (i1 if cy else i0)[1], (i1 if cx else i0)[0]]
    k = torch.ones(1, 1, 3, 3, 3, dtype=torch.float64)
    cnt = torch.nn.functional.conv3d(torch.ones(1, 1, *shape, dtype=torch.float64), k, padding=1)[0, 0]

    def bmean(v):
        return torch.nn.functional.conv3d(v[None, None], k, padding=1)[0, 0] / cnt

    mu_m, mu_s = bmean(m), bmean(Is)
    sd_m = torch.sqrt(torch.clamp(bmean(m * m) - mu_m ** 2, min=0))
    sd_s = torch.sqrt(torch.clamp(bmean(Is * Is) - mu_s ** 2, min=0))
    a = sd_m / sd_s
    f = a * Is + (mu_m - a * mu_s)
    loss = ((m - f) ** 2).sum()
    loss.backward()
    assert float(loss.detach()) == pytest.approx(O.ssd_loss(I_m, I_s, r, half), rel=1e-12)
    np.testing.assert_allclose(g, rt.grad.numpy(), rtol=1e-8, atol=1e-8 * np.abs(g).max())


def test_smoothing_order_variant_linearity():
    """Sec. 2.1 order (r + G*dr) against A1's (G*(r + dr)): the Gaussian is linear,
    so the two differ by exactly r - G*r; with r = 0 they coincide."""
    rng = np.random.default_rng(31)
    shape = (6, 8, 10)
    I_m = rng.normal(0.0, 100.0, shape)
    I_s = 0.9 * np.roll(I_m, 1, axis=2) + 5.0
    r = rng.normal(0.0, 0.5, (3,) + shape)
    pa = O.Params(patch=(3, 3, 3), sigma=1.0, levels=1, iters=[1])
    pb = O.Params(patch=(3, 3, 3), sigma=1.0, levels=1, iters=[1], smooth_mode=1)
    ra, dra, _, _ = O.iteration(I_m, I_s, r, pa)
    rb, drb, _, _ = O.iteration(I_m, I_s, r, pb)
    np.testing.assert_array_equal(dra, drb)
    np.testing.assert_allclose(rb - ra, r - O.gaussian_smooth_field(r, 1.0), atol=1e-12)
    z = np.zeros_like(r)
    np.testing.assert_allclose(O.iteration(I_m, I_s, z, pa)[0], O.iteration(I_m, I_s, z, pb)[0], atol=1e-12)


# ------------------------------------------- direct pins of three building blocks

def test_box_sum_against_brute_force():
    """Eq. (3)'s truncated patch sum against a scalar loop over the clipped box,
    with an anisotropic half size (hx, hy, hz) so that a swapped axis fails."""
    X = _rng(41).normal(size=(5, 6, 7))           # [nz][ny][nx]
    half = (2, 1, 0)                               # (hx, hy, hz)
    got = O.box_sum(X, half)
    nz, ny, nx = X.shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                s = 0.0
                for zz in range(max(0, z - half[2]), min(nz, z + half[2] + 1)):
                    for yy in range(max(0, y - half[1]), min(ny, y + half[1] + 1)):
                        for xx in range(max(0, x - half[0]), min(nx, x + half[0] + 1)):
                            s += X[zz, yy, xx]
                assert got[z, y, x] == pytest.approx(s, abs=1e-12)


def test_warp_coord_gradient_is_the_derivative_of_the_warp():
    """d I_m(x + r) / d r_a equals the oracle's coordinate gradient: inside a
    trilinear cell the warp is linear along each axis, so a central difference
    of the warp with a step that stays in the cell is exact (up to rounding); an
    axis whose sample is clamped has derivative 0."""
    rng = _rng(43)
    I_m = rng.normal(size=(6, 7, 8)) * 100.0
    shape = I_m.shape
    # fractions in [0.2, 0.8] and sample positions strictly inside the volume
    base = rng.integers(-1, 2, size=(3,) + shape).astype(np.float64)
    r = base + rng.uniform(0.2, 0.8, size=(3,) + shape)
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    pos = [x + r[0], y + r[1], z + r[2]]
    inside = np.ones(shape, bool)
    for a, n in enumerate((shape[2], shape[1], shape[0])):
        inside &= (pos[a] > 0.0) & (pos[a] < n - 1)
    assert inside.sum() > 100
    g = O.warp_coord_gradient(I_m, r)
    eps = 1e-3
    for a in range(3):
        rp, rm = r.copy(), r.copy()
        rp[a] += eps
        rm[a] -= eps
        fd = (O.warp(I_m, rp) - O.warp(I_m, rm)) / (2.0 * eps)
        np.testing.assert_allclose(g[a][inside], fd[inside], rtol=1e-6, atol=1e-6)
    # a sample pushed far outside along x is clamped there: zero x derivative
    rc = r.copy()
    rc[0] = 100.0
    assert np.all(O.warp_coord_gradient(I_m, rc)[0] == 0.0)


def test_build_pyramid_shapes_means_and_worked_example():
    """Sec. 2.3's pyramid (reading R13): each level halves every extent rounding
    up; for even extents a level's mean equals the finer level's (2x2x2 means of
    full cells); the 2x2x2 volume 0..7 becomes its mean 3.5."""
    img = _rng(47).normal(size=(8, 12, 16))
    pyr = O.build_pyramid(img, 3)
    assert [p.shape for p in pyr] == [(8, 12, 16), (4, 6, 8), (2, 3, 4)]
    assert pyr[1].mean() == pytest.approx(img.mean(), abs=1e-12)
    assert pyr[2].mean() == pytest.approx(img.mean(), abs=1e-12)
    assert pyr[1][1, 2, 3] == pytest.approx(img[2:4, 4:6, 6:8].mean(), abs=1e-12)
    small = O.build_pyramid(np.arange(8.0).reshape(2, 2, 2), 2)
    assert small[1].shape == (1, 1, 1) and small[1][0, 0, 0] == 3.5
    odd = O.build_pyramid(np.arange(27.0).reshape(3, 3, 3), 2)[1]
    assert odd.shape == (2, 2, 2)
    assert odd[1, 1, 1] == 26.0                       # a partial corner cell: its one voxel
    assert odd[0, 0, 1] == pytest.approx(np.mean([2, 5, 11, 14]), abs=1e-12)
