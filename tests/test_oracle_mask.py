"""Pins of the oracle's mask and fill (Eqs. 7-10, Sec. 2.3, Algorithm A1 step 2).

Closed forms (a two-neighbour weighted mean that fixes the sign and the h^2
scale of Eq. 10; the median ratio of an affine CBCT), invariants (a filled
value is a convex combination of known values; known values never change; a
constant known a is reproduced; Jacobi propagation reaches distance 3p in x
and p in z after p passes of the 7 x 7 x 3 box), special cases (xi = 0
everywhere reduces to the unmasked correction; an affine CBCT is recovered
exactly through the fill) and the stated readings (R17-R20).
"""
import math

import numpy as np
import pytest

from oracle import disc_oracle as O


def test_two_neighbour_weights_closed_form():
    h = 40.0
    I_s = np.array([[[100.0, 100.0, 100.0 + 2 * h]]])    # [nz=1][ny=1][nx=3]
    a = np.array([[[1.0, 0.0, 2.0]]])
    b = np.array([[[10.0, 0.0, 20.0]]])
    xi = np.array([[[False, True, False]]])
    fa, fb, st = O.fill_coefficients(a, b, xi, I_s, h, (3, 3, 1), 4)
    w = math.exp(-4.0)                                   # (2h / h)^2 = 4
    assert fa[0, 0, 1] == pytest.approx((1.0 + 2.0 * w) / (1.0 + w), rel=1e-14)
    assert fb[0, 0, 1] == pytest.approx((10.0 + 20.0 * w) / (1.0 + w), rel=1e-14)
    assert st.tolist() == [[[0, 1, 0]]]
    # a neighbour darker by 2h weighs the same as one brighter by 2h
    I_s2 = np.array([[[100.0, 100.0, 100.0 - 2 * h]]])
    fa2, _, _ = O.fill_coefficients(a, b, xi, I_s2, h, (3, 3, 1), 4)
    assert fa2[0, 0, 1] == pytest.approx(fa[0, 0, 1], rel=1e-14)


def test_fill_invariants_random():
    rng = np.random.default_rng(3)
    shape = (5, 9, 11)
    I_s = rng.normal(0.0, 60.0, shape)
    a = rng.uniform(0.5, 2.0, shape)
    b = rng.uniform(-50.0, 50.0, shape)
    xi = rng.random(shape) < 0.6
    fa, fb, st = O.fill_coefficients(a, b, xi, I_s, 50.0, (3, 3, 1), 50)
    known = ~xi
    assert np.array_equal(fa[known], a[known]) and np.array_equal(fb[known], b[known])
    assert np.all(st[known] == 0) and np.all(st[xi] >= 1)          # all reachable here
    lo, hi = a[known].min(), a[known].max()
    assert np.all(fa[xi] >= lo - 1e-12) and np.all(fa[xi] <= hi + 1e-12)
    # a constant known a (and b) is reproduced wherever it is interpolated
    fa_c, fb_c, _ = O.fill_coefficients(np.full(shape, 1.7), np.full(shape, -3.0), xi, I_s, 50.0,
                                        (3, 3, 1), 50)
    np.testing.assert_allclose(fa_c, 1.7, rtol=1e-14)
    np.testing.assert_allclose(fb_c, -3.0, rtol=1e-14)


def test_jacobi_propagation_distance():
    # x: half width 3 -> the voxel at distance d is filled in pass ceil(d / 3)
    n = 20
    xi = np.ones((1, 1, n), bool)
    xi[0, 0, 0] = False
    a = np.ones((1, 1, n))
    _, _, st = O.fill_coefficients(a, a, xi, np.zeros((1, 1, n)), 50.0, (3, 3, 1), 100)
    assert st[0, 0].tolist() == [0] + [math.ceil(d / 3) for d in range(1, n)]
    # z: half width 1 -> pass d
    xi = np.ones((n, 1, 1), bool)
    xi[0] = False
    a = np.ones((n, 1, 1))
    _, _, st = O.fill_coefficients(a, a, xi, np.zeros((n, 1, 1)), 50.0, (3, 3, 1), 100)
    assert st[:, 0, 0].tolist() == list(range(n))
    # the pass cap leaves the far voxels unfilled, with a = b = 0
    fa, _, st = O.fill_coefficients(np.full((n, 1, 1), 2.0), a, xi, np.zeros((n, 1, 1)), 50.0, (3, 3, 1), 5)
    assert st[:, 0, 0].tolist() == list(range(6)) + [-1] * (n - 6)
    assert np.all(fa[6:] == 0.0) and np.all(fa[:6] == 2.0)


@pytest.mark.parametrize("t_half,seed", [((3, 3, 1), 0), ((1, 2, 2), 1), ((0, 1, 3), 2)])
def test_fill_front_is_box_dilation(t_half, seed):
    """A voxel is filled in the first pass after one of its box neighbours is
    known, so the voxels known after pass p are the p-fold dilation of the
    unmasked voxels by the box T (scipy's binary dilation, an independent
    routine): the stamps are the dilation levels, capped by the pass limit."""
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    shape = (9, 13, 17)
    xi = rng.random(shape) < 0.93                      # mostly masked: deep fronts
    xi[4, 6, 8] = False
    known = ~xi
    tx, ty, tz = t_half
    box = np.ones((2 * tz + 1, 2 * ty + 1, 2 * tx + 1), bool)
    level = np.where(known, 0, -1)
    cur = known.copy()
    for p in range(1, 7):
        nxt = ndimage.binary_dilation(cur, structure=box)
        level[nxt & ~cur] = p
        cur = nxt
    a = rng.normal(size=shape)
    _, _, st = O.fill_coefficients(a, a, xi, rng.normal(0.0, 30.0, shape), 50.0, t_half, 6)
    np.testing.assert_array_equal(st, level)


def test_nothing_known_and_exponent_cap():
    shape = (2, 3, 4)
    xi = np.ones(shape, bool)
    fa, fb, st = O.fill_coefficients(np.ones(shape), np.ones(shape), xi, np.zeros(shape), 50.0)
    assert np.all(st == -1) and np.all(fa == 0.0) and np.all(fb == 0.0)
    # neighbours 1e4 HU away still weigh exp(-80) each (R20): the voxel is filled
    I_s = np.array([[[0.0, 1e4, 0.0]]])
    a = np.array([[[3.0, 0.0, 5.0]]])
    xi = np.array([[[False, True, False]]])
    fa, _, st = O.fill_coefficients(a, a, xi, I_s, 50.0, (3, 3, 1), 4)
    assert st[0, 0, 1] == 1 and fa[0, 0, 1] == pytest.approx(4.0, rel=1e-14)


def test_mask_xi_conditions():
    m = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    I_s = np.array([0.0, 250.0, 0.0, 0.0, 0.0, -199.0])
    a = np.array([1.0, 1.0, 0.4, 1.6, 1.0, 1.0])
    valid = np.array([True, True, True, True, False, True])
    xi = O.mask_xi(m, I_s, a, valid, 200.0, 0.5, 1.5)
    assert xi.tolist() == [False, True, True, True, True, False]


def test_ratio_median_of_affine_cbct():
    rng = np.random.default_rng(5)
    I_m = rng.normal(0.0, 100.0, (6, 10, 12))
    for alpha in (0.8, -1.25, 2.0):
        I_s = alpha * I_m + 37.0
        assert O.ratio_median(I_m, I_s, (1, 1, 1)) == pytest.approx(1.0 / abs(alpha), rel=1e-12)


def _noisy_pair(shape, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    I_m = 300.0 * np.sin(0.3 * x + 0.2 * y) + 100.0 * np.cos(0.4 * z) + rng.normal(0.0, 20.0, shape)
    return I_m


def test_xi_zero_reduces_to_unmasked_correction():
    shape = (6, 10, 12)
    I_m = _noisy_pair(shape, 1)
    rng = np.random.default_rng(2)
    I_s = 0.7 * I_m + rng.normal(0.0, 25.0, shape) + 40.0
    off = O.MaskState(hu0=np.inf, a_min=0.0, a_max=np.inf)
    f, xi, st = O.correct_masked(I_m, I_s, (1, 1, 1), off, 50.0)
    assert not xi.any() and np.all(st == 0)
    np.testing.assert_array_equal(f, O.correct(I_m, I_s, (1, 1, 1)))


def test_affine_cbct_recovered_through_the_fill():
    """I_s = alpha I_m + beta: every known voxel has a = 1/alpha, b = -beta/alpha
    (Appendix A), so the fill reproduces them and I'_s = I_m everywhere, also
    at the masked voxels (here masked by a narrow a range and a HU0 band)."""
    shape = (6, 10, 12)
    I_m = _noisy_pair(shape, 4)
    alpha, beta = 0.8, 30.0
    I_s = alpha * I_m + beta
    # a = 1.25 everywhere: a_max just above keeps all voxels but the HU0 band
    mask = O.MaskState(hu0=60.0, a_min=0.0, a_max=1.2500001)
    f, xi, st = O.correct_masked(I_m, I_s, (1, 1, 1), mask, 50.0, (3, 3, 1), 64)
    assert xi.any() and (~xi).any() and np.all(st >= 0)
    np.testing.assert_allclose(f, I_m, rtol=0, atol=1e-9 * np.abs(I_m).max())


def test_register_mask_off_equals_plain():
    shape = (8, 12, 16)
    I_m = _noisy_pair(shape, 7)
    rng = np.random.default_rng(8)
    I_s = 0.9 * np.roll(I_m, 1, axis=2) + rng.normal(0.0, 10.0, shape)
    p = O.Params(patch=(3, 3, 3), sigma=1.0, levels=1, iters=[3])
    r0 = O.register(I_m, I_s, p)
    pm = O.Params(patch=(3, 3, 3), sigma=1.0, levels=1, iters=[3], mask_mode=1, hu0_factor=1e9,
                  a_lo=0.0, a_hi=1e9)
    np.testing.assert_array_equal(O.register(I_m, I_s, pm), r0)
    # and with a real mask the field stays finite and differs
    pm2 = O.Params(patch=(3, 3, 3), sigma=1.0, levels=1, iters=[3], mask_mode=1)
    r2 = O.register(I_m, I_s, pm2)
    assert np.all(np.isfinite(r2)) and not np.array_equal(r2, r0)


def test_ratio_median_ignores_constant_ct_patches():
    """Reading R18: patches where the CT is constant (a = 0 whatever the CBCT) do
    not enter the median, even when they are most of the volume."""
    rng = np.random.default_rng(6)
    shape = (6, 10, 24)
    I_m = np.full(shape, -1000.0)
    I_m[:, :, 16:] = rng.normal(0.0, 100.0, (6, 10, 8))     # textured third; the rest flat
    I_s = 0.5 * I_m + rng.normal(0.0, 1e-3, shape) * (I_m == -1000.0) + 10.0
    assert O.ratio_median(I_m, I_s, (1, 1, 1)) == pytest.approx(2.0, rel=1e-6)
