"""The bulk-tensor-copy (TMA) form of the moment pass against the plain-load form.

Both forms run the same arithmetic in the same order; only the way the z march
reads global memory differs (bulk tensor copies into shared memory, with zeros
outside the volume, versus per-thread loads with bounds tests).  Their outputs
must therefore be bitwise equal.  The DISC_SW_NO_TMA test switch selects the plain-load form at
planning time.  The TMA form needs nx a multiple of 4 and extents of at least
one staging box (48 x 30 voxels for patch 11 in iteration mode); the shapes
below meet that with ragged tiles in x, y and z.  (The per-kernel oracle
tests include shapes that take the TMA form as well.)  The TMA form also takes
the first planes of each chunk's z window, which only enter the z sums, as
bursts of bulk copies; the shapes include chunks at the volume's start (fewer
warm-up planes), a volume shorter than the patch, and warm-ups longer than one
burst.
"""

import numpy as np
import pytest

from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, empty, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _NoTma():
    from paper_1204_6295_b300 import disc
    return disc.test_switches(disc.SW_NO_TMA)


def _Wide():
    """The wide-tile iteration pass (32 x 32 tiles, balanced z shares) at any size."""
    from paper_1204_6295_b300 import disc
    return disc.test_switches(disc.SW_WIDE_ANY)


def _SeparateWarp():
    """The next iteration's warp in a kernel of its own, after the Gaussian, at every level."""
    from paper_1204_6295_b300 import disc
    return disc.test_switches(disc.SW_SEPARATE_WARP)


def _FusedWarp():
    """The next iteration's warp inside the Gaussian xy pass at every level."""
    from paper_1204_6295_b300 import disc
    return disc.test_switches(disc.SW_FUSED_WARP)


CASES = [
    ((20, 40, 64), 3),      # (nz, ny, nx), patch
    ((33, 47, 100), 11),    # ragged in all three axes
    ((9, 64, 48), 15),      # patch wider than the chunk, exact box width
    ((40, 31, 52), 7),
    ((17, 52, 96), 5),
    # patch 15 on 40 planes: chunks starting at z >= 8 have 14 warm-up planes,
    # more than the staging area holds (12 boxes in iteration mode, 8 in the
    # static pass), so the warm-up burst runs in two rounds
    ((40, 36, 48), 15),
]


def _inputs(shape, patch, seed):
    ct = ct_like(shape, seed, noise=15.0)
    cbct = ct_like(shape, seed + 1, noise=25.0)
    r = phantom.smooth_random_field(shape, seed + 2, amp=2.5).astype(np.float32)
    return ct, cbct, r


@pytest.mark.parametrize("shape,patch", CASES)
@pytest.mark.parametrize("force_mode", [0, 1])
def test_force_update_bitwise(disc, shape, patch, force_mode):
    P = (patch,) * 3
    ct, cbct, r = _inputs(shape, patch, 40 + patch)
    qs_m = disc.qscale(float(np.abs(ct).max()), P)
    qs_s = disc.qscale(float(np.abs(cbct).max()), P)
    Im, Is, rd = dev(ct), dev(cbct), dev(r)
    zs = empty(*shape)
    m = empty(*shape)
    disc.k_static_norm(Is, zs, P, qs_s)
    disc.k_warp(Im, rd, m)
    outs = []
    for form in ("tma", "plain", "wide"):
        u = empty(3, *shape)
        d = empty(*shape)
        norms = empty(2).double()
        ctx = {"plain": _NoTma, "wide": _Wide}.get(form)
        if ctx:
            with ctx():
                disc.k_force_update(m, zs, rd, u, P, qs_m, d_out=d, norms_out=norms, force_mode=force_mode)
        else:
            disc.k_force_update(m, zs, rd, u, P, qs_m, d_out=d, norms_out=norms, force_mode=force_mode)
        outs.append((host(u), host(d), host(norms)))
    disc.k_check_error()
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0][0], o[0])
        np.testing.assert_array_equal(outs[0][1], o[1])
        # the norm partials are per CTA, and the forms split the volume differently
        np.testing.assert_allclose(outs[0][2], o[2], rtol=1e-6)


@pytest.mark.parametrize("shape,patch", CASES[:3] + CASES[-1:])
def test_static_norm_bitwise(disc, shape, patch):
    P = (patch,) * 3
    _, cbct, _ = _inputs(shape, patch, 7)
    qs = disc.qscale(float(np.abs(cbct).max()), P)
    Is = dev(cbct)
    z1, z2 = empty(*shape), empty(*shape)
    disc.k_static_norm(Is, z1, P, qs)
    with _NoTma():
        disc.k_static_norm(Is, z2, P, qs)
    np.testing.assert_array_equal(host(z1), host(z2))


@pytest.mark.parametrize("shape,patch", [((20, 40, 64), 3), ((18, 34, 56), 9)])
def test_ssd_bitwise(disc, shape, patch):
    P = (patch,) * 3
    ct, cbct, r = _inputs(shape, patch, 90)
    qs_m = disc.qscale(float(np.abs(ct).max()), P)
    qs_s = disc.qscale(float(np.abs(cbct).max()), P)
    Im, Is, rd = dev(ct), dev(cbct), dev(r)
    zs = empty(*shape)
    disc.k_static_norm(Is, zs, P, qs_s)
    res = []
    for plain in (False, True):
        g = empty(3, *shape)
        loss = empty(1).double()
        if plain:
            with _NoTma():
                disc.k_ssd_grad(Im, zs, rd, g, P, qs_m, loss_out=loss)
        else:
            disc.k_ssd_grad(Im, zs, rd, g, P, qs_m, loss_out=loss)
        res.append((host(g), host(loss)))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_allclose(res[0][1], res[1][1], rtol=1e-6)   # per-CTA partial sums


def test_registration_bitwise(disc):
    """A whole two-level schedule through the context: the TMA form, plain loads,
    and the wide-tile pass at the finest level."""
    shape = (32, 64, 64)
    ct, cbct, _ = _inputs(shape, 9, 11)
    fields = []
    for form in ("tma", "plain", "wide", "separate_warp", "fused_warp"):
        def run():
            reg = disc.Registration(patch=(9, 9, 9), sigma=1.0, levels=2, iters=(6, 5))
            reg.set_images(dev(ct), dev(cbct))
            reg.iterate(-1)
            out = empty(3, *shape)
            reg.get_field(out)
            return host(out)
        ctx = {"plain": _NoTma, "wide": _Wide, "separate_warp": _SeparateWarp, "fused_warp": _FusedWarp}.get(form)
        if ctx:
            with ctx():
                fields.append(run())
        else:
            fields.append(run())
    for f in fields[1:]:
        np.testing.assert_array_equal(fields[0], f)


# Shapes on which the planner itself picks the wide-tile pass (enough (tile,
# plane) pairs for its wave): ragged in y and z, patch 11 and 15, Thirion and
# double force, against the plain-load 32 x 16 pass.
@pytest.mark.parametrize("shape,patch,force_mode", [((150, 250, 256), 11, 0), ((131, 200, 192), 15, 1)])
def test_planner_wide_pass_bitwise(disc, shape, patch, force_mode):
    P = (patch,) * 3
    ct, cbct, r = _inputs(shape, patch, 60 + patch)
    qs_m = disc.qscale(float(np.abs(ct).max()), P)
    qs_s = disc.qscale(float(np.abs(cbct).max()), P)
    Im, Is, rd = dev(ct), dev(cbct), dev(r)
    zs, m = empty(*shape), empty(*shape)
    disc.k_static_norm(Is, zs, P, qs_s)
    disc.k_warp(Im, rd, m)
    outs = []
    for plain in (False, True):
        u, d, norms = empty(3, *shape), empty(*shape), empty(2).double()
        if plain:
            with _NoTma():
                disc.k_force_update(m, zs, rd, u, P, qs_m, d_out=d, norms_out=norms, force_mode=force_mode)
        else:
            disc.k_force_update(m, zs, rd, u, P, qs_m, d_out=d, norms_out=norms, force_mode=force_mode)
        outs.append((host(u), host(d), host(norms)))
    disc.k_check_error()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_allclose(outs[0][2], outs[1][2], rtol=1e-6)


# The SSD adjoint pass on wide tiles: where the planner picks it (large volumes)
# and forced on a small ragged one, against the plain-load 32 x 16 pass; the
# gradient bit for bit, the loss to the partial sums' rounding.
@pytest.mark.parametrize("shape,patch,wide_any", [((150, 250, 256), 11, False), ((131, 200, 192), 15, False),
                                                  ((33, 70, 96), 5, True)])
def test_wide_adjoint_pass_bitwise(disc, shape, patch, wide_any):
    P = (patch,) * 3
    ct, cbct, r = _inputs(shape, patch, 80 + patch)
    qs_m = disc.qscale(float(np.abs(ct).max()), P)
    qs_s = disc.qscale(float(np.abs(cbct).max()), P)
    Im, Is, rd = dev(ct), dev(cbct), dev(r)
    zs = empty(*shape)
    disc.k_static_norm(Is, zs, P, qs_s)
    res = []
    for plain in (False, True):
        g = empty(3, *shape)
        loss = empty(1).double()
        with (_NoTma() if plain else disc.test_switches(disc.SW_WIDE_ANY if wide_any else 0)):
            disc.k_ssd_grad(Im, zs, rd, g, P, qs_m, loss_out=loss)
            g2 = empty(3, *shape)
            disc.k_ssd_grad(Im, zs, rd, g2, P, qs_m)        # no loss: no partials
        np.testing.assert_array_equal(host(g), host(g2))
        res.append((host(g), host(loss)))
    disc.k_check_error()
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_allclose(res[0][1], res[1][1], rtol=1e-6)


def test_wide_mask_pass_bitwise(disc):
    """The mask pass of Eqs. 5-7 on wide tiles (and the ratio pass of a_m at set-up)
    inside a masked two-level registration, against the plain-load 32 x 16 pass:
    the same mask constants and the same field, bit for bit."""
    pair = phantom.ellipsoid_pair(96, 64, 40, seed=81)
    kw = dict(patch=(7, 7, 7), sigma=1.0, levels=2, iters=(3, 3), mask_mode=1)
    out = []
    for ctx in (lambda: disc.test_switches(disc.SW_WIDE_ANY), _NoTma):
        with ctx():
            with disc.Registration(**kw) as reg:
                reg.set_images(pair.ct, pair.cbct)
                consts = reg.mask_constants()
                reg.iterate(-1)
                out.append((consts, reg.get_field()))
    disc.k_check_error()
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_bounded_wait_reports_timeout_and_device_stays_usable(disc):
    """A copy group armed for 16 bytes more than its copies deliver (the
    DISC_SW_TMA_STALL test switch of the iteration pass) never completes: the wait gives
    up after about a second, the CTA drains and returns, the context reports
    DISC_ERR_TIMEOUT and then refuses further work, and a new context on the same
    device runs normally."""
    pair = phantom.ellipsoid_pair(64, 48, 16, seed=3)
    kw = dict(patch=(3, 3, 3), sigma=1.0, levels=1, iters=(1,))
    with disc.test_switches(disc.SW_TMA_STALL):
        reg = disc.Registration(**kw)
        reg.set_images(pair.ct, pair.cbct)          # the static pass is not stalled
        with pytest.raises(disc.DiscError) as e:
            reg.iterate(-1)
        assert e.value.status == 6                  # DISC_ERR_TIMEOUT
        with pytest.raises(disc.DiscError) as e2:
            reg.iterate(-1)
        assert e2.value.status == 3                 # DISC_ERR_STATE: the failure is sticky
        reg.close()
    with disc.Registration(**kw) as reg:
        reg.set_images(pair.ct, pair.cbct)
        done, _ = reg.iterate(-1)
        r = reg.get_field()
    assert done == 1 and np.isfinite(r).all() and np.abs(r).max() > 0
    disc.k_check_error()
