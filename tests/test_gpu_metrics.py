"""Parity of the evaluation metrics (Sec. 2.4.3, Eq. 11) with the oracle.

The GPU takes every integer decision (histogram bin, non-maximum test,
threshold) in float32 with the oracle's operation order, so the histograms and
the Canny edge maps must agree exactly; the entropies are summed in double in
different orders (NMI to 1e-12).
"""
import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, empty, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


@pytest.mark.parametrize("bins", [2, 16, 64, 128])
def test_nmi_matches_oracle(disc, bins):
    a = ct_like((12, 40, 56), 1, noise=20.0)
    b = (0.8 * a + np.random.default_rng(2).normal(0.0, 40.0, a.shape)).astype(np.float32)
    out = empty(1).double()
    disc.k_nmi(dev(a), dev(b), out, bins)
    assert host(out)[0] == pytest.approx(O.nmi(a, b, bins), abs=1e-12)
    disc.k_nmi(dev(a), dev(a), out, bins)
    assert host(out)[0] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("shape,sigma,t_low,t_high", [
    ((3, 48, 64), 1.0, 0.4, 0.2),
    ((2, 37, 70), 0.5, 0.3, 0.3),
    ((4, 64, 33), 2.0, 0.4, 0.1),
])
def test_canny_matches_oracle_exactly(disc, shape, sigma, t_low, t_high):
    import torch
    img = ct_like(shape, 3, noise=15.0)
    e = torch.empty(shape, dtype=torch.uint8, device="cuda")
    disc.k_canny(dev(img), e, sigma, t_low, t_high)
    got = e.cpu().numpy().astype(bool)
    ref = O.canny(img, sigma, t_low, t_high)
    assert ref.any() and (~ref).any()
    np.testing.assert_array_equal(got, ref)


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
    ref = O.edge_rmse(O.canny(a), O.canny(b))
    assert ref > 0 and host(out)[0] == pytest.approx(ref, rel=1e-12)
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
