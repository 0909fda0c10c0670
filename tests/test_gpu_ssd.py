"""Differentiable form: SSD loss and its adjoint gradient on the GPU against the
FP64 oracle (whose adjoint is itself pinned to central differences and to an
independent torch-autograd formulation), central finite differences on a
32^3 crop of the head-and-neck pair, and the torch.autograd.Function wrapper."""
import math

import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, empty, host, rel_err

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3     # gradient: relative to finite differences / the FP64 adjoint
LOSS_TOL = 1e-5


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _prepare(disc, ct, cbct, patch):
    import torch
    qs_s = disc.qscale(float(np.abs(cbct).max()), patch)
    qs_m = disc.qscale(float(np.abs(ct).max()), patch)
    zs = empty(*ct.shape)
    disc.k_static_norm(dev(cbct), zs, patch, qs_s)
    return dev(ct), zs, qs_m


def _gpu_loss_grad(disc, ct, cbct, r, patch):
    import torch
    ct_d, zs, qs = _prepare(disc, ct, cbct, patch)
    r_d = dev(r)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    loss2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = empty(3, *ct.shape)
    disc.k_ssd_loss(ct_d, zs, r_d, loss, patch, qs)
    disc.k_ssd_grad(ct_d, zs, r_d, grad, patch, qs, loss_out=loss2)
    torch.cuda.synchronize()
    # the same d^2 terms, grouped by the adjoint pass's CTAs
    assert float(loss2.item()) == pytest.approx(float(loss.item()), rel=1e-6)
    return float(loss.item()), host(grad)


@pytest.mark.parametrize("shape,patch", [((12, 14, 16), (3, 3, 3)), ((13, 35, 40), (5, 5, 5)),
                                         ((9, 20, 70), (7, 7, 7)), ((1, 6, 9), (3, 3, 3))])
def test_ssd_loss_and_adjoint_match_oracle(disc, shape, patch):
    ct = ct_like(shape, 41)
    cbct = (ct_like(shape, 42, noise=20.0) * 0.8 + 30.0).astype(np.float32)
    r = phantom.smooth_random_field(shape, 43, amp=1.7) if min(shape) > 1 else \
        phantom.random_field(shape, 43, amp=1.2)
    half = tuple((p - 1) // 2 for p in patch)
    loss, grad = _gpu_loss_grad(disc, ct, cbct, r, patch)
    assert loss == pytest.approx(O.ssd_loss(ct, cbct, r, half), rel=LOSS_TOL)
    ref = O.ssd_grad(ct, cbct, r, half)
    assert rel_err(grad, ref) <= GRAD_TOL, rel_err(grad, ref)


@pytest.fixture(scope="module")
def headneck_crop():
    p = phantom.head_neck_pair()
    sl = (slice(48, 80), slice(112, 144), slice(112, 144))
    ct = np.ascontiguousarray(p.ct[sl])
    cbct = np.ascontiguousarray(p.cbct[sl])
    u = np.ascontiguousarray(p.u_true[(slice(None),) + sl])
    return ct, cbct, u


def test_ssd_gradient_matches_central_differences_on_headneck_crop(disc, headneck_crop):
    """32^3 crop of the head-and-neck pair, patch 11^3, eps = 1e-3 voxel (FP64 loss)."""
    ct, cbct, u = headneck_crop
    patch, half = (11, 11, 11), (5, 5, 5)
    r = (0.6 * u).astype(np.float32)
    _, grad = _gpu_loss_grad(disc, ct, cbct, r, patch)
    eps = 1e-3
    rng = np.random.default_rng(44)
    fd_vals, g_vals = [], []
    nz, ny, nx = ct.shape
    while len(fd_vals) < 24:
        c = int(rng.integers(0, 3))
        z, y, x = (int(rng.integers(1, n - 1)) for n in (nz, ny, nx))
        pos = (x, y, z)[c] + float(r[c, z, y, x])
        frac = pos - math.floor(pos)
        if frac < 2 * eps or frac > 1 - 2 * eps:
            continue          # trilinear kink within the difference stencil
        rp = r.astype(np.float64).copy()
        rp[c, z, y, x] += eps
        rm = r.astype(np.float64).copy()
        rm[c, z, y, x] -= eps
        fd = (O.ssd_loss(ct, cbct, rp, half) - O.ssd_loss(ct, cbct, rm, half)) / (2 * eps)
        fd_vals.append(fd)
        g_vals.append(grad[c, z, y, x])
    fd_vals, g_vals = np.array(fd_vals), np.array(g_vals)
    assert np.abs(g_vals - fd_vals).max() <= GRAD_TOL * np.abs(fd_vals).max(), (g_vals, fd_vals)


def test_autograd_function_uses_the_adjoint_kernels(disc, headneck_crop):
    import torch
    from paper_1204_6295_b300.ssd import SSDLoss
    ct, cbct, u = headneck_crop
    patch = (5, 5, 5)
    model = SSDLoss(dev(ct), dev(cbct), patch)
    r = dev(0.5 * u).requires_grad_(True)
    loss = model(r)
    (2.5 * loss).backward()
    grad = empty(3, *ct.shape)
    disc.k_ssd_grad(model.ct, model.zs, r.detach(), grad, patch, model.qs)
    np.testing.assert_allclose(host(r.grad), 2.5 * host(grad), rtol=1e-6, atol=0)
    assert float(loss.item()) == pytest.approx(O.ssd_loss(ct, cbct, 0.5 * u.astype(np.float64)
                                                          .astype(np.float32), (2, 2, 2)), rel=LOSS_TOL)


def test_ssd_full_size_gradient_at_sampled_voxels(disc):
    """256x256x128 pair, patch 11^3: the whole-volume gradient at sampled voxels equals
    the oracle's on a crop holding every voxel the sample depends on."""
    p = phantom.head_neck_pair()
    patch, half, H = (11, 11, 11), (5, 5, 5), 5
    r = (0.7 * p.u_true).astype(np.float32)
    loss, grad = _gpu_loss_grad(disc, p.ct, p.cbct, r, patch)
    assert np.isfinite(loss) and np.isfinite(grad).all()
    nz, ny, nx = p.ct.shape
    halo = 2 * H + 2 + int(np.ceil(np.abs(r).max())) + 1
    samples = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (64, 128, 128), (5, 200, 31), (100, 17, 240),
               (64, 0, 100)]
    for (z, y, x) in samples:
        z0, z1 = max(0, z - halo), min(nz, z + halo + 1)
        y0, y1 = max(0, y - halo), min(ny, y + halo + 1)
        x0, x1 = max(0, x - halo), min(nx, x + halo + 1)
        sl = (slice(z0, z1), slice(y0, y1), slice(x0, x1))
        ref = O.ssd_grad(p.ct[sl], p.cbct[sl], r[(slice(None),) + sl], half)[:, z - z0, y - y0, x - x0]
        got = grad[:, z, y, x]
        scale = max(np.abs(ref).max(), 1e-6 * np.abs(grad).max())
        assert np.abs(got - ref).max() <= GRAD_TOL * scale, ((z, y, x), got, ref)


@pytest.mark.parametrize("level", [0, 1])
def test_context_ssd_equals_kernel_level_calls(disc, level):
    """disc_ssd on a registration context's own pyramid level (its CT, its CBCT
    normalisation zs and fixed-point scale) equals the kernel-level calls on the
    same level's images bit for bit, for device and host buffers."""
    import torch
    shape, patch = (20, 36, 48), (5, 5, 5)
    ct = ct_like(shape, 51)
    cbct = (ct_like(shape, 52, noise=20.0) * 0.8 + 30.0).astype(np.float32)
    kw = dict(patch=patch, sigma=1.0, levels=2, iters=(2, 2), global_shift=0)
    with disc.Registration(**kw) as reg:
        reg.set_images(dev(ct), dev(cbct))
        ct_l, cb_l = dev(ct), dev(cbct)
        if level == 1:
            nz, ny, nx = [(s + 1) // 2 for s in shape]
            a, b = empty(nz, ny, nx), empty(nz, ny, nx)
            disc.k_downsample2(ct_l, a)
            disc.k_downsample2(cb_l, b)
            ct_l, cb_l = a, b
        lshape = tuple(ct_l.shape)
        r = phantom.smooth_random_field(lshape, 53 + level, amp=1.5).astype(np.float32)
        g_dev = empty(3, *lshape)
        loss_dev = reg.ssd(level, dev(r), g_dev)
        g_host = np.empty((3,) + lshape, np.float32)
        loss_host = reg.ssd(level, r, g_host)
        loss_only = reg.ssd(level, dev(r))
        # the registration state is untouched: it still runs its schedule
        assert reg.iterate(-1)[0] == 4
    qs_m = disc.qscale(float(np.abs(ct).max()), patch)      # the finest level's scales serve every level
    qs_s = disc.qscale(float(np.abs(cbct).max()), patch)
    zs = empty(*lshape)
    disc.k_static_norm(cb_l, zs, patch, qs_s)
    g_ref = empty(3, *lshape)
    l_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    l_ref2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    disc.k_ssd_grad(ct_l, zs, dev(r), g_ref, patch, qs_m, loss_out=l_ref)
    disc.k_ssd_loss(ct_l, zs, dev(r), l_ref2, patch, qs_m)
    np.testing.assert_array_equal(host(g_dev), host(g_ref))
    np.testing.assert_array_equal(g_host, host(g_ref).astype(np.float32))
    assert loss_dev == float(l_ref.item()) and loss_host == loss_dev
    assert loss_only == float(l_ref2.item())
