"""Pins of the oracle's evaluation metrics (Sec. 2.4.3; readings R21, R22).

NMI: identity and exact affine maps give 1, independent two-level images give
0 in closed form, symmetry.  Canny: a constant image has no edges; a step
whose central difference peaks on one column gives exactly that column;
hysteresis keeps a weak edge joined to a strong one and drops an isolated weak
one; thresholds scale with the slice's largest gradient.  Eq. (11) on edge
maps with a known number of differing pixels.
"""
import math

import numpy as np
import pytest

from oracle import disc_oracle as O


def test_nmi_special_cases():
    rng = np.random.default_rng(1)
    A = rng.integers(0, 16, size=(4, 8, 8)).astype(np.float32)
    assert O.nmi(A, A, 16) == pytest.approx(1.0, abs=1e-12)
    assert O.nmi(A, 3.0 * A - 7.0, 16) == pytest.approx(1.0, abs=1e-12)    # bins map one to one
    # two independent two-level images: I = 0 exactly
    a = np.array([0, 0, 1, 1] * 4, np.float32)
    b = np.array([0, 1, 0, 1] * 4, np.float32)
    assert O.nmi(a, b, 2) == pytest.approx(0.0, abs=1e-12)
    # a perfect two-level dependence through a permutation of levels: still 1
    assert O.nmi(a, 1.0 - a, 2) == pytest.approx(1.0, abs=1e-12)
    B = rng.normal(size=A.shape).astype(np.float32)
    assert O.nmi(A, B, 16) == pytest.approx(O.nmi(B, A, 16), abs=1e-12)
    assert O.nmi(np.zeros(10, np.float32), np.ones(10, np.float32), 8) == 1.0


def _step(shape, col, lo=0.0, hi=100.0):
    img = np.full(shape, lo, np.float32)
    img[..., col + 1:] = hi
    img[..., col] = 0.5 * (lo + hi)       # central difference peaks on this column only
    return img


def test_canny_constant_and_single_step():
    assert not O.canny(np.full((2, 12, 16), 7.0, np.float32)).any()
    E = O.canny(_step((2, 16, 24), 10), sigma=0.5)
    assert np.all(E[..., 10])                                    # the step column, every row
    assert not np.any(np.delete(E, 10, axis=2))                  # and nothing else


def test_canny_hysteresis():
    """A vertical edge whose height falls from strong to weak along its length
    stays whole; a separate weak edge of the weak height is dropped."""
    ny, nx = 24, 40
    img = np.zeros((1, ny, nx), np.float32)
    h = np.linspace(100.0, 30.0, ny).astype(np.float32)[:, None]   # step height along the edge
    img[0, :, 11:] = h
    img[0, :, 10:11] = 0.5 * h
    img[0, :, 31:] += 30.0                                      # separate weak step
    img[0, :, 30] += 15.0
    E = O.canny(img, sigma=0.5, t_low=0.4, t_high=0.5)[0]
    assert np.all(E[:, 10])                                      # strong and joined weak part
    assert not np.any(E[:, 30])                                  # isolated weak edge dropped
    # with a low enough high threshold the second edge becomes strong too
    E2 = O.canny(img, sigma=0.5, t_low=0.4, t_high=0.2)[0]
    assert np.all(E2[:, 30])


def test_edge_rmse_closed_form():
    E1 = np.zeros((3, 5, 7), bool)
    E2 = E1.copy()
    E2[1, 2, 3] = E2[0, 0, 0] = E2[2, 4, 6] = True
    assert O.edge_rmse(E1, E2) == pytest.approx(math.sqrt(3 / E1.size), rel=1e-15)
    assert O.edge_rmse(E2, E2) == 0.0


def test_nmi_histogram_matches_numpy_histogram2d():
    """The joint histogram of reading R21 is numpy's histogram2d over each image's
    [min, max] with `bins` equal bins (a library special case), so the NMI built
    from histogram2d's counts is the oracle's."""
    rng = np.random.default_rng(5)
    A = rng.normal(0.0, 300.0, size=(5, 20, 30))
    B = 0.5 * A + rng.normal(0.0, 100.0, size=A.shape)
    for bins in (2, 7, 64):
        h, _, _ = np.histogram2d(A.ravel(), B.ravel(), bins=bins,
                                 range=[[A.min(), A.max()], [B.min(), B.max()]])
        p = h / A.size
        pa, pb = p.sum(1), p.sum(0)
        ent = lambda q: -(q[q > 0] * np.log(q[q > 0])).sum()
        ha, hb, hab = ent(pa), ent(pb), ent(p.ravel())
        assert O.nmi(A, B, bins) == pytest.approx(2.0 * (ha + hb - hab) / (ha + hb), abs=1e-13)


def test_canny_diagonal_step_is_one_pixel_wide():
    """A step across the line x + y = c has its gradient along the 45-degree
    diagonal: non-maximum suppression along that diagonal (reading R22) leaves
    a line one pixel wide in the direction of the gradient, on the step."""
    ny, nx = 32, 32
    y, x = np.mgrid[0:ny, 0:nx]
    img = np.where(x + y > 31, 100.0, 0.0)[None]
    E = O.canny(img, sigma=1.0)[0]
    inner = E[6:-6, 6:-6]
    yy, xx = np.nonzero(inner)
    assert yy.size > 0
    s = (xx + 6) + (yy + 6)
    assert set(np.unique(s)) <= {31, 32}          # on the step
    # one pixel wide along the gradient (the diagonal): never both of a pixel and its (+1, +1) neighbour
    assert not np.any(E[:-1, :-1] & E[1:, 1:])
