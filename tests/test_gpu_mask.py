"""Parity of the mask-and-fill path (Eqs. 7-10) with the FP64 oracle.

Per step, the oracle is fed the GPU's own float32 inputs of that step (R16).
Decisions taken in floating point (xi of Eq. 7) are compared away from their
thresholds: where |m - I_s| or a lies within a relative 1e-4 of HU0, a_min or
a_max the two precisions may decide differently, and the fill comparison then
takes the GPU's own decisions as its input.  The fill decision itself (a pass
fills a voxel iff it has a known neighbour, reading R20) does not depend on
the precision, so the pass stamps must agree exactly.
"""
import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, empty, host, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _pair(shape, seed):
    """CT-like moving image; CBCT = affine copy + noise + a bright streak block."""
    ct = ct_like(shape, seed, noise=15.0).astype(np.float64)
    rng = np.random.default_rng(seed + 1)
    cbct = 0.85 * ct + 25.0 + rng.normal(0.0, 20.0, shape)
    nz, ny, nx = shape
    cbct[nz // 3: nz // 3 + 4, ny // 4: ny // 2, nx // 5: nx // 2] += 450.0     # artifact
    return ct.astype(np.float32), cbct.astype(np.float32)


def _static(disc, Is, patch):
    qs = disc.qscale(float(np.abs(Is).max()), patch)
    zs, sd = empty(*Is.shape), empty(*Is.shape)
    disc.k_static_stats(dev(Is), zs, sd, patch, qs)
    return zs, sd


SHAPES = [((20, 40, 64), (5, 5, 5)),      # takes the TMA box pass
          ((13, 37, 70), (7, 5, 3))]      # generic box pass, ragged tiles


@pytest.mark.parametrize("shape,patch", SHAPES)
def test_static_stats_std(disc, shape, patch):
    _, Is = _pair(shape, 1)
    zs, sd = _static(disc, Is, patch)
    qs = disc.qscale(float(np.abs(Is).max()), patch)
    zs2 = empty(*shape)
    disc.k_static_norm(dev(Is), zs2, patch, qs)
    np.testing.assert_array_equal(host(zs), host(zs2))
    half = tuple((p - 1) // 2 for p in patch)
    E1, E2 = O.patch_moments(Is.astype(np.float64), half)
    ref = O.patch_std(E1, E2)
    assert rel_err(host(sd), ref) <= TOL


@pytest.mark.parametrize("shape,patch", SHAPES)
def test_ratio_median(disc, shape, patch):
    ct, Is = _pair(shape, 2)
    zs, sd = _static(disc, Is, patch)
    qs = disc.qscale(float(np.abs(ct).max()), patch)
    a = empty(*shape)
    med = empty(1).double()
    disc.k_ratio_median(dev(ct), zs, sd, a, med, patch, qs)
    ag = host(a)
    half = tuple((p - 1) // 2 for p in patch)
    ref_a, _ = O.intensity_coefficients(ct, Is, half)
    ok = ag >= 0
    assert ok.mean() > 0.9
    assert rel_err(ag[ok], ref_a[ok]) <= 1e-4
    # the median of the GPU's own values: exact order statistics
    assert host(med)[0] == np.median(ag[ok].astype(np.float32).astype(np.float64))
    assert host(med)[0] == pytest.approx(O.ratio_median(ct, Is, half), rel=1e-4)


def _near(x, t, rel=1e-4):
    return np.abs(x - t) <= rel * max(abs(t), 1.0)


FILLS = [((7, 7, 3), 32),                # Sec. 2.3's box T, every masked voxel reached
         ((15, 9, 5), 32),               # wide x span: the known-voxel bits cross mask words
         ((3, 3, 1), 2),                 # a pass cap that leaves voxels unfilled
         ((1, 3, 3), 1)]                 # a box one voxel wide in x


@pytest.mark.parametrize("fill_t,passes", FILLS)
@pytest.mark.parametrize("shape,patch", SHAPES)
def test_mask_and_fill(disc, shape, patch, fill_t, passes):
    ct, Is = _pair(shape, 3)
    r = phantom.smooth_random_field(shape, 4, amp=1.5).astype(np.float32)
    zs, sd = _static(disc, Is, patch)
    qs = disc.qscale(float(np.abs(ct).max()), patch)
    m = empty(*shape)
    disc.k_warp(dev(ct), dev(r), m)
    a_w = empty(*shape)
    med = empty(1).double()
    disc.k_ratio_median(dev(ct), zs, sd, a_w, med, patch, qs)
    a_m = float(host(med)[0])
    hu0, a_min, a_max = 150.0, 0.5 * a_m, 1.5 * a_m
    import torch
    a, b, d = empty(*shape), empty(*shape), empty(*shape)
    stamp = torch.empty(shape, dtype=torch.int32, device="cuda")
    left = torch.zeros(1, dtype=torch.int32, device="cuda")
    disc.k_correct_masked(m, dev(Is), zs, sd, a, b, d, stamp, patch, qs, hu0, a_min, a_max,
                          fill_h=50.0, fill_t=fill_t, fill_passes=passes, remaining_out=left)
    disc.k_check_error()
    m64, Is64 = host(m), Is.astype(np.float64)
    st = stamp.cpu().numpy()
    half = tuple((p - 1) // 2 for p in patch)
    # Eqs. 5-6 and Eq. 7 from the GPU's m
    a_o, b_o = O.intensity_coefficients(m64, Is64, half)
    ES, ES2 = O.patch_moments(Is64, half)
    valid = np.maximum(ES2 - ES * ES, 0.0) > 1e-6
    xi_o = O.mask_xi(m64, Is64, a_o, valid, hu0, a_min, a_max)
    xi_g = st != 0
    assert xi_g.any() and (~xi_g).any()
    ambiguous = _near(np.abs(m64 - Is64), hu0) | _near(a_o, a_min) | _near(a_o, a_max)
    assert np.array_equal(xi_g[~ambiguous], xi_o[~ambiguous])
    # the fill from the GPU's own decisions: stamps exact, values to float32 accuracy
    fa, fb, fst = O.fill_coefficients(a_o, b_o, xi_g, Is64, 50.0, tuple((t - 1) // 2 for t in fill_t), passes)
    np.testing.assert_array_equal(st, fst)
    assert int(left.cpu()[0]) == int((fst < 0).sum())
    if passes < 32:
        assert (fst < 0).any()                   # the cap left some voxels unfilled
    assert rel_err(host(a), fa) <= 1e-4
    # a of Eq. 5 where it is not filled and both patch variances are well away
    # from the quantisation (> 1 HU^2): 1e-5 relative, voxel by voxel
    EM, EM2 = O.patch_moments(m64, half)
    good = (fst == 0) & (np.maximum(EM2 - EM * EM, 0.0) > 1.0) & (np.maximum(ES2 - ES * ES, 0.0) > 1.0)
    assert good.mean() > 0.5
    ag = host(a)
    assert np.all(np.abs(ag[good] - fa[good]) <= 1e-5 * np.abs(fa[good]))
    # b = E(M) - a E(S) cancels: its error scales with the intensities, not with b
    assert np.abs(host(b) - fb).max() <= 1e-4 * np.abs(fa * Is64).max()
    f_ref = fa * Is64 + fb
    assert rel_err(m64 + host(d), f_ref) <= 1e-5


@pytest.mark.parametrize("force_mode", [0, 1])
def test_force_from_d_matches_oracle_and_box_pass(disc, force_mode):
    shape, patch = (18, 33, 64), (5, 5, 5)
    ct, Is = _pair(shape, 5)
    r = phantom.smooth_random_field(shape, 6, amp=2.0).astype(np.float32)
    zs, _ = _static(disc, Is, patch)
    qs = disc.qscale(float(np.abs(ct).max()), patch)
    import torch
    u1, m, d = empty(3, *shape), empty(*shape), empty(*shape)
    disc.k_pass_a(dev(ct), zs, dev(r), u1, patch, qs, m_out=m, d_out=d, force_mode=force_mode)
    u2 = empty(3, *shape)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    disc.k_force(m, d, dev(r), u2, norms_out=norms, force_mode=force_mode)
    # the same arithmetic as the box pass's force stage: bitwise equal
    np.testing.assert_array_equal(host(u1), host(u2))
    m64 = host(m)
    dr_ref = O.force(m64, m64 + host(d), force_mode)
    dr_g = host(u2) - r.astype(np.float64)
    assert np.abs(dr_g - dr_ref).max() <= TOL * max(np.abs(dr_ref).max(), 1e-3)
    n = host(norms)
    assert n[0] == pytest.approx(np.sqrt((dr_ref ** 2).sum(0)).sum(), rel=1e-5)


def test_registration_mask_with_nothing_masked_equals_plain(disc):
    shape = (24, 48, 64)
    ct, Is = _pair(shape, 7)                      # the mask is opened wide below
    fields = []
    for kw in (dict(mask_mode=0), dict(mask_mode=1, hu0_factor=1e9, a_lo=0.0, a_hi=1e9)):
        reg = disc.Registration(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(4, 3), **kw)
        reg.set_images(dev(ct), dev(Is))
        reg.iterate(-1)
        out = empty(3, *shape)
        reg.get_field(out)
        fields.append(host(out))
    np.testing.assert_array_equal(fields[0], fields[1])


BAND = 1e-4      # relative margin within which float32 and float64 may decide xi differently


def _oracle_masked_run(ct, Is, p):
    """The oracle's masked registration (as O.register), also returning the smallest
    relative margin of any xi decision (Eq. 7) of the run: | |m - I_s| - HU0 | / HU0
    and |a - a_min| / a_min, |a - a_max| / a_max where a is defined."""
    I_m, I_s = ct.astype(np.float64), Is.astype(np.float64)
    I_s, dhu = O.global_shift(I_m, I_s)
    a_m = O.ratio_median(I_m, I_s, p.half, p.var_floor)
    mask = O.MaskState(p.hu0_factor * abs(dhu), p.a_lo * a_m, p.a_hi * a_m)
    pm, ps = O.build_pyramid(I_m, p.levels), O.build_pyramid(I_s, p.levels)
    r = np.zeros((3,) + pm[-1].shape)
    worst, masked, in_band, decisions = 1.0, [], 0, 0
    for lev in range(p.levels - 1, -1, -1):
        for _ in range(p.iters[p.levels - 1 - lev]):
            m = O.warp(pm[lev], r)
            a, _ = O.intensity_coefficients(m, ps[lev], p.half, p.var_floor)
            ES, ES2 = O.patch_moments(ps[lev], p.half)
            valid = np.maximum(ES2 - ES * ES, 0.0) > p.var_floor
            hm = np.abs(np.abs(m - ps[lev]) - mask.hu0) / mask.hu0
            am = np.minimum(np.abs(a - mask.a_min) / mask.a_min, np.abs(a - mask.a_max) / mask.a_max)[valid]
            worst = min(worst, hm.min(), am.min() if am.size else 1.0)
            in_band += int(np.count_nonzero(hm <= BAND) + np.count_nonzero(am <= BAND))
            decisions += hm.size
            masked.append(O.mask_xi(m, ps[lev], a, valid, mask.hu0, mask.a_min, mask.a_max).mean())
            r, _, _, _ = O.iteration(pm[lev], ps[lev], r, p, mask)
        if lev > 0:
            r = O.upsample_field2(r, pm[lev - 1].shape)
    return r, worst, masked, mask, (in_band, decisions)


def test_registration_masked_matches_oracle_at_full_bars(disc):
    """A masked registration whose every xi decision (at every voxel and
    iteration of the oracle's run) lies further than BAND from its threshold:
    float32 and float64 then take the same decisions, and the field must meet
    the end-to-end bars (1e-2 voxel max, 1e-4 mean) everywhere.  The thresholds'
    factors are stepped from the paper's (2, 0.5, 1.5) until the oracle's run has
    no decision inside the band."""
    shape = (12, 24, 40)
    ct, Is = _pair(shape, 9)
    kw = dict(patch=(3, 3, 3), sigma=1.0, levels=2, iters=(5, 4), mask_mode=1)
    for t in range(16):
        f = dict(hu0_factor=2.0 * 1.013 ** t, a_lo=0.5 * 0.987 ** t, a_hi=1.5 * 1.011 ** t)
        p = O.Params(patch=kw["patch"], sigma=kw["sigma"], levels=kw["levels"], iters=list(kw["iters"]),
                     mask_mode=1, **f)
        ref, worst, masked, mask, _ = _oracle_masked_run(ct, Is, p)
        if worst > BAND:
            break
    assert worst > BAND, worst
    assert min(masked) > 0.01                      # the mask and the fill are exercised
    reg = disc.Registration(**kw, **f)
    reg.set_images(dev(ct), dev(Is))
    hu0, a_m = reg.mask_constants()
    reg.iterate(-1)
    out = empty(3, *shape)
    reg.get_field(out)
    reg.close()
    disc.k_check_error()
    assert hu0 == pytest.approx(mask.hu0, rel=1e-5)
    assert a_m * f["a_lo"] == pytest.approx(mask.a_min, rel=1e-5)
    diff = np.sqrt(((host(out) - ref) ** 2).sum(0))
    assert diff.max() <= 1e-2 and diff.mean() <= 1e-4, (diff.max(), diff.mean())


def test_registration_masked_with_threshold_ties(disc):
    """The paper's threshold factors on a larger pair, where some xi decisions of
    the run lie within BAND of their thresholds: the two precisions may decide
    those differently.  Checks that such decisions are rare (under 0.01% of the
    run's decisions lie in the band) and that the field stays within a
    documented looser bar (mean 1e-3, 99.9th percentile 1e-2 voxel)."""
    shape = (16, 32, 48)
    ct, Is = _pair(shape, 9)
    kw = dict(patch=(3, 3, 3), sigma=1.0, levels=2, iters=(6, 5), mask_mode=1)
    reg = disc.Registration(**kw)
    reg.set_images(dev(ct), dev(Is))
    hu0, a_m = reg.mask_constants()
    reg.iterate(-1)
    out = empty(3, *shape)
    reg.get_field(out)
    reg.close()
    disc.k_check_error()
    p = O.Params(patch=(3, 3, 3), sigma=1.0, levels=2, iters=[6, 5], mask_mode=1)
    ref = O.register(ct, Is, p)
    ref2, worst, _, _, (in_band, decisions) = _oracle_masked_run(ct, Is, p)
    np.testing.assert_array_equal(ref, ref2)      # the replay is the oracle's registration
    assert worst <= BAND and 0 < in_band <= 1e-4 * decisions, (worst, in_band, decisions)
    _, dhu = O.global_shift(ct, Is)
    assert hu0 == pytest.approx(2.0 * abs(dhu), rel=1e-5)
    Is_sh = Is.astype(np.float64) + dhu
    assert a_m == pytest.approx(O.ratio_median(ct, Is_sh, (1, 1, 1)), rel=1e-4)
    diff = np.sqrt(((host(out) - ref) ** 2).sum(0))
    assert np.mean(diff) <= 1e-3
    assert np.quantile(diff, 0.999) <= 1e-2
