"""Parity of the evaluation metrics (Sec. 2.4.3, Eq. 11) with the FP64 oracle.

The oracle takes every decision (histogram bin, gradient sector, non-maximum
test, thresholds) in float64; the GPU takes them in float32.  A GPU decision
may differ from the oracle's only where the float64 margin of that decision is
within float32 rounding:
  - NMI: a value whose float64 bin coordinate lies within BIN_EPS of a bin
    boundary may fall in either bin; the NMI may move by at most the effect of
    moving those voxels (a bound on the entropy change per voxel), and must
    agree to 1e-12 when there is none;
  - Canny: with d = DELTA max|slice|, a bound on the float32 error of the
    smoothed slice, its gradient and magnitude, a comparison whose float64
    margin is within d (scaled by the comparison's coefficients) may go either
    way.  Hysteresis is monotone in the candidate and strong sets, so the GPU's
    edge map must contain the edges of the surely-taken decisions and lie
    inside the edges of the possibly-taken ones; the pixels between the two
    are the excused ones, reported and required to be under 1% of the slice.
"""
import math

import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, empty, host

pytestmark = pytest.mark.gpu

DELTA = 4e-5          # float32 error bound of S, gx, gy, M relative to max|slice| (about 10x the estimate)
BIN_EPS = 1e-6        # float32 error bound of the bin coordinate, per bin


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


def _ambiguous_bins(X, bins):
    X = np.asarray(X, np.float64).ravel()
    mn, mx = X.min(), X.max()
    if mx == mn:
        return np.zeros(X.shape, bool)
    t = (X - mn) * bins / (mx - mn)
    frac = np.abs(t - np.round(t))
    return (frac <= BIN_EPS * bins) & (t > 0.5) & (t < bins - 0.5)


def _nmi_tolerance(a, b, bins):
    """1e-12 plus the largest NMI change the ambiguous voxels can cause."""
    k = int(np.count_nonzero(_ambiguous_bins(a, bins) | _ambiguous_bins(b, bins)))
    n = a.size
    ia, ib = O.nmi_bins(a, bins), O.nmi_bins(b, bins)

    def ent(idx):
        c = np.bincount(idx, minlength=bins) / n
        c = c[c > 0]
        return -(c * np.log(c)).sum()

    hs = ent(ia) + ent(ib)
    if hs == 0.0:
        return k, 1e-12
    # one voxel moved to another bin changes each entropy by at most 2 (ln n + 1) / n
    return k, 1e-12 + 12.0 * (math.log(n) + 1.0) * k / (n * hs)


@pytest.mark.parametrize("bins", [2, 16, 64, 128])
def test_nmi_matches_oracle(disc, bins):
    a = ct_like((12, 40, 56), 1, noise=20.0)
    b = (0.8 * a + np.random.default_rng(2).normal(0.0, 40.0, a.shape)).astype(np.float32)
    out = empty(1).double()
    disc.k_nmi(dev(a), dev(b), out, bins)
    k, tol = _nmi_tolerance(a, b, bins)
    assert abs(host(out)[0] - O.nmi(a, b, bins)) <= tol, (k, tol)
    assert k <= a.size // 1000
    disc.k_nmi(dev(a), dev(a), out, bins)
    assert host(out)[0] == pytest.approx(1.0, abs=1e-12)


def test_nmi_exact_away_from_bin_boundaries(disc):
    """Values at bin centres: no decision is ambiguous, so the NMI agrees to 1e-12."""
    rng = np.random.default_rng(3)
    bins = 32
    ja = rng.integers(0, bins, size=(6, 30, 40))
    jb = np.clip(ja + rng.integers(-2, 3, size=ja.shape), 0, bins - 1)
    ja[0, 0, 0], ja[0, 0, 1] = 0, bins - 1                 # span the full range: centres map to bins
    jb[0, 0, 0], jb[0, 0, 1] = 0, bins - 1
    a = (-500.0 + 25.0 * (ja + 0.5)).astype(np.float32)   # min, max at the first and last centres
    b = (100.0 + 7.5 * (jb + 0.5)).astype(np.float32)
    assert not _ambiguous_bins(a, bins).any() and not _ambiguous_bins(b, bins).any()
    out = empty(1).double()
    disc.k_nmi(dev(a), dev(b), out, bins)
    assert host(out)[0] == pytest.approx(O.nmi(a, b, bins), abs=1e-12)


def _canny_bounds(img, sigma, t_low, t_high):
    """Edge maps of the surely-taken and the possibly-taken decisions (see the module text)."""
    img = np.asarray(img, np.float64)
    lo_e = np.zeros(img.shape, bool)
    hi_e = np.zeros(img.shape, bool)
    for z in range(img.shape[0]):
        P = img[z]
        q = O.canny_slice(P, sigma, t_low, t_high)
        d = DELTA * max(np.abs(P).max(), 1e-30)
        M, gx, gy, sec = q["M"], q["gx"], q["gy"], q["sector"]
        ax, ay = np.abs(gx), np.abs(gy)
        t1, t2 = O.CANNY_TAN1, O.CANNY_TAN2
        amb_sec = ((np.abs(ay - t1 * ax) <= d * (1 + t1)) | (np.abs(ay - t2 * ax) <= d * (1 + t2))
                   | (ax <= d) | (ay <= d))
        sure_k = np.ones((4,) + M.shape, bool)
        poss_k = np.ones((4,) + M.shape, bool)
        for k in range(4):
            n1, n2 = q["n1"][k], q["n2"][k]
            sure_k[k] = (M - q["floor"] > d) & (M - n1 > 2 * d) & (M - n2 > 2 * d)
            poss_k[k] = (M - q["floor"] >= -d) & (M - n1 >= -2 * d) & (M - n2 >= -2 * d)
        own_sure = np.take_along_axis(sure_k, sec[None], 0)[0]
        own_poss = np.take_along_axis(poss_k, sec[None], 0)[0]
        keep_sure = np.where(amb_sec, sure_k.all(0), own_sure)
        keep_poss = np.where(amb_sec, poss_k.any(0), own_poss)
        dh = d * (1 + t_high)                 # M and t_high max(M) both carry the error
        dl = d * (1 + t_low * t_high)
        strong_sure = keep_sure & (M - q["hi"] > dh)
        strong_poss = keep_poss & (M - q["hi"] >= -dh)
        cand_sure = keep_sure & (M - q["lo"] > dl)
        cand_poss = keep_poss & (M - q["lo"] >= -dl)
        lo_e[z] = O.canny_hysteresis(cand_sure, strong_sure)
        hi_e[z] = O.canny_hysteresis(cand_poss, strong_poss)
    return lo_e, hi_e


@pytest.mark.parametrize("shape,sigma,t_low,t_high", [
    ((3, 48, 64), 1.0, 0.4, 0.2),
    ((2, 37, 70), 0.5, 0.3, 0.3),
    ((4, 64, 33), 2.0, 0.4, 0.1),
])
def test_canny_matches_oracle_within_rounding(disc, shape, sigma, t_low, t_high):
    import torch
    img = ct_like(shape, 3, noise=15.0)
    e = torch.empty(shape, dtype=torch.uint8, device="cuda")
    disc.k_canny(dev(img), e, sigma, t_low, t_high)
    got = e.cpu().numpy().astype(bool)
    ref = O.canny(img, sigma, t_low, t_high)
    assert ref.any() and (~ref).any()
    lo_e, hi_e = _canny_bounds(img, sigma, t_low, t_high)
    assert np.all(lo_e <= ref) and np.all(ref <= hi_e)          # the bounds bracket the oracle
    assert np.all(lo_e <= got), np.argwhere(lo_e & ~got)[:5]    # every sure edge found
    assert np.all(got <= hi_e), np.argwhere(got & ~hi_e)[:5]    # no edge beyond rounding
    excused = int(np.count_nonzero(hi_e & ~lo_e))
    differ = int(np.count_nonzero(got != ref))
    print(f"canny {shape}: {differ} pixels differ from float64, {excused} excused by rounding margins")
    assert excused <= 0.01 * got.size


def test_edge_rmse_and_registration_metrics(disc):
    import torch
    shape = (4, 40, 48)
    a = ct_like(shape, 5, noise=10.0)
    b = np.roll(a, 2, axis=2)
    ea = torch.empty(shape, dtype=torch.uint8, device="cuda")
    eb = torch.empty(shape, dtype=torch.uint8, device="cuda")
    disc.k_canny(dev(a), ea, 1.0, 0.4, 0.2)
    disc.k_canny(dev(b), eb, 1.0, 0.4, 0.2)
    out = empty(1).double()
    disc.k_edge_rmse(ea, eb, out)
    # Eq. (11) exactly on the GPU's own edge maps
    ga, gb = ea.cpu().numpy().astype(bool), eb.cpu().numpy().astype(bool)
    assert host(out)[0] == pytest.approx(O.edge_rmse(ga, gb), rel=1e-12)
    # and within the excused pixels of the float64 edge maps' RMSE
    la, ha = _canny_bounds(a, 1.0, 0.4, 0.2)
    lb, hb = _canny_bounds(b, 1.0, 0.4, 0.2)
    amb = (ha & ~la) | (hb & ~lb)
    ref = O.edge_rmse(O.canny(a), O.canny(b))
    n = a.size
    assert ref > 0
    assert abs(host(out)[0] ** 2 - ref ** 2) <= np.count_nonzero(amb) / n + 1e-12
    # the context's metrics: warped CT against corrected CBCT, before and after registering
    p = phantom.ellipsoid_pair(48, 40, 24, seed=5)
    with disc.Registration(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(20, 20)) as reg:
        reg.set_images(p.ct, p.cbct)
        nmi0, rmse0 = reg.metrics()
        reg.iterate(-1)
        nmi1, rmse1 = reg.metrics()
        m = O.warp(p.ct, reg.get_field()).astype(np.float32)
        f = reg.get_corrected()
    assert 0.0 <= nmi0 <= 1.0 and 0.0 <= nmi1 <= 1.0
    assert nmi1 > nmi0 and rmse1 < rmse0                       # registration improved both
    assert nmi1 == pytest.approx(O.nmi(m, f, 64), abs=1e-3)    # m from the oracle's warp (float64)
