"""The averages of the correction coefficients a, b (Eqs. 5-6; Sec. 3.4 plots
them over the iterations) through disc_get_correction_means, against the FP64
oracle on the GPU's own field (reading R16: the oracle is fed the GPU's float32
state of the step).
"""
import numpy as np
import pytest

from oracle import disc_oracle as O

from gpu_util import ct_like, dev, empty, host

pytestmark = pytest.mark.gpu

SHAPE = (14, 30, 44)
PATCH = (3, 3, 3)
BAND = 1e-4


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _pair(seed):
    ct = ct_like(SHAPE, seed, noise=15.0).astype(np.float64)
    rng = np.random.default_rng(seed + 1)
    cbct = 0.85 * ct + 25.0 + rng.normal(0.0, 20.0, SHAPE)
    nz, ny, nx = SHAPE
    cbct[nz // 3: nz // 3 + 4, ny // 4: ny // 2, nx // 5: nx // 2] += 450.0
    return ct.astype(np.float32), cbct.astype(np.float32)


def _run(disc, ct, cbct, iters, **kw):
    reg = disc.Registration(patch=PATCH, sigma=1.0, levels=1, iters=(iters,), **kw)
    reg.set_images(dev(ct), dev(cbct))
    means = [reg.correction_means()]
    reg.iterate(-1)
    means.append(reg.correction_means())
    out = empty(3, *SHAPE)
    reg.get_field(out)
    consts = reg.mask_constants() if kw.get("mask_mode") else None
    reg.close()
    disc.k_check_error()
    return means, host(out), consts


def test_correction_means_unmasked_match_oracle(disc):
    ct, cbct = _pair(3)
    means, r, _ = _run(disc, ct, cbct, 4)
    I_m = ct.astype(np.float64)
    I_s, _ = O.global_shift(I_m, cbct.astype(np.float64))
    half = tuple((p - 1) // 2 for p in PATCH)
    ES, ES2 = O.patch_moments(I_s, half)
    valid = np.maximum(ES2 - ES * ES, 0.0) > 1e-6
    scale = float(np.abs(I_s).max())
    for (ma, mb, n), field in zip(means, (np.zeros_like(r), r)):
        m = O.warp(I_m, field)
        a, b = O.intensity_coefficients(m, I_s, half)
        assert n == int(valid.sum())
        assert ma == pytest.approx(a[valid].mean(), rel=1e-5)
        assert abs(mb - b[valid].mean()) <= 1e-5 * scale
    # the field moved, so the means of the two calls differ
    assert means[0] != means[1]


def test_correction_means_mask_wide_open_equals_unmasked(disc):
    ct, cbct = _pair(5)
    plain, r0, _ = _run(disc, ct, cbct, 3)
    opened, r1, _ = _run(disc, ct, cbct, 3, mask_mode=1, hu0_factor=1e9, a_lo=0.0, a_hi=1e9)
    np.testing.assert_array_equal(r0, r1)
    assert plain == opened


def test_correction_means_masked_match_oracle(disc):
    """With the mask on: a, b after the mask (Eq. 7) and the fill (Eqs. 8-10),
    averaged over the voxels known or filled.  The thresholds are stepped from
    the paper's factors until no xi decision on the GPU's warped image lies
    within BAND of its threshold, so that both precisions decide alike."""
    ct, cbct = _pair(7)
    half = tuple((p - 1) // 2 for p in PATCH)
    I_m = ct.astype(np.float64)
    I_s, _ = O.global_shift(I_m, cbct.astype(np.float64))
    ES, ES2 = O.patch_moments(I_s, half)
    valid = np.maximum(ES2 - ES * ES, 0.0) > 1e-6
    p = O.Params()
    for t in range(16):
        f = dict(hu0_factor=2.0 * 1.013 ** t, a_lo=0.5 * 0.987 ** t, a_hi=1.5 * 1.011 ** t)
        means, r, (hu0, a_m) = _run(disc, ct, cbct, 3, mask_mode=1, **f)
        cases = []
        worst = 1.0
        for field, got in zip((np.zeros_like(r), r), means):
            m = O.warp(I_m, field)
            a, b = O.intensity_coefficients(m, I_s, half)
            a_min, a_max = f["a_lo"] * a_m, f["a_hi"] * a_m
            hm = np.abs(np.abs(m - I_s) - hu0) / hu0
            am = np.minimum(np.abs(a - a_min) / a_min, np.abs(a - a_max) / a_max)[valid]
            worst = min(worst, hm.min(), am.min() if am.size else 1.0)
            xi = O.mask_xi(m, I_s, a, valid, hu0, a_min, a_max)
            cases.append((a, b, xi, got))
        if worst > BAND:
            break
    assert worst > BAND, worst
    scale = float(np.abs(I_s).max())
    for a, b, xi, (ma, mb, n) in cases:
        assert 0.01 < xi.mean() < 0.9                 # the mask and the fill are exercised
        fa, fb, stamp = O.fill_coefficients(a, b, xi, I_s, p.fill_h, p.fill_half, p.fill_passes)
        known = stamp >= 0
        assert n == int(known.sum())
        assert ma == pytest.approx(fa[known].mean(), rel=1e-5)
        assert abs(mb - fb[known].mean()) <= 1e-5 * scale


def test_correction_means_errors(disc):
    reg = disc.Registration(patch=PATCH, sigma=1.0, levels=1, iters=(1,))
    with pytest.raises(disc.DiscError) as e:
        reg.correction_means()                   # no images yet
    assert e.value.status == 3
    reg.close()
