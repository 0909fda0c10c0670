"""Plain FP64 CPU oracle for the DISC hot path (Zhen et al., arXiv 1204.6295).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The CUDA library never
calls it and shares no code with it.

Every function follows one passage of the paper, in the paper's notation, with
numpy float64 arrays and no blocking, fusion or reordering beyond what the
definition states.  Where the paper is silent or garbled the reading used is
stated in the docstring (readings R1..R22, listed with their reasons in the
design notes of the repository).

Layout: images are ``[nz][ny][nx]`` (x fastest); fields are ``[3][nz][ny][nx]``
with components (x, y, z), in voxel units of the level they live on.

Roles (Sec. 2.2): the moving image ``I_m`` is the planning CT, the static image
``I_s`` is the CBCT; the field ``r`` relates them by ``I_m(x + r(x)) = I_s(x)``
(Sec. 2.1).

Pins: every function here is checked in ``tests/test_oracle_pins.py``,
``tests/test_oracle_mask.py`` and ``tests/test_oracle_metrics.py`` against
brute force, closed forms, library special cases or invariants.  A function
without an independent pin would be noted as "parity unpinned" below (none at
present).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

AXES = ("x", "y", "z")          # field component order
ARRAY_AXIS = {0: 2, 1: 1, 2: 0}  # field component -> numpy axis of [nz][ny][nx]

FORCE_THIRION = 0
FORCE_DOUBLE = 1


# ---------------------------------------------------------------------------
# Sec. 2.3, first paragraph; Algorithm A1, first line: global intensity shift
# ---------------------------------------------------------------------------

def global_shift(I_m, I_s):
    """Shift the CBCT by the constant dHU that equalises the two image means.

    Sec. 2.3: a constant shift of the CBCT intensity so that the mean
    intensities of CT and CBCT agree.  Returns (shifted I_s, dHU).
    """
    I_m = np.asarray(I_m, np.float64)
    I_s = np.asarray(I_s, np.float64)
    dHU = I_m.mean() - I_s.mean()
    return I_s + dHU, dHU


# ---------------------------------------------------------------------------
# Sec. 2.3, multi-scale strategy; Algorithm A1 "down-sample" / "up-sample"
# Reading R13: 2x2x2 mean down-sampling, cell-centred trilinear up-sampling.
# ---------------------------------------------------------------------------

def level_dims(dims, levels):
    """Grid sizes (nx, ny, nz) of each pyramid level, finest first.

    Each coarser level has ceil(n/2) voxels per axis (reading R13).
    """
    out = [tuple(int(d) for d in dims)]
    for _ in range(1, levels):
        out.append(tuple((d + 1) // 2 for d in out[-1]))
    return out


def downsample2(img):
    """Sec. 2.3 multi-scale strategy (reading R13): mean over each 2x2x2 cell; a
    partial last cell averages its in-bounds voxels."""
    img = np.asarray(img, np.float64)
    nz, ny, nx = img.shape
    cz, cy, cx = (nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2
    acc = np.zeros((cz, cy, cx))
    cnt = np.zeros((cz, cy, cx))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                sub = img[dz::2, dy::2, dx::2]
                acc[:sub.shape[0], :sub.shape[1], :sub.shape[2]] += sub
                cnt[:sub.shape[0], :sub.shape[1], :sub.shape[2]] += 1.0
    return acc / cnt


def _clamped_linear_coords(n_fine, n_coarse):
    """Reading R13 (cell-centred up-sampling): index pairs and weights mapping fine
    voxel i to coarse position (i - 0.5)/2, clamped."""
    pos = (np.arange(n_fine, dtype=np.float64) - 0.5) / 2.0
    pos = np.clip(pos, 0.0, n_coarse - 1)
    i0 = np.floor(pos).astype(np.int64)
    t = pos - i0
    i1 = np.minimum(i0 + 1, n_coarse - 1)
    return i0, i1, t


def upsample_field2(r_coarse, fine_shape):
    """Coarse field -> fine field: trilinear at (x - 0.5)/2, values doubled.

    The field is in voxel units, and a coarse voxel spans two fine voxels, so
    the displacement magnitude doubles (reading R13).
    """
    r_coarse = np.asarray(r_coarse, np.float64)
    nzf, nyf, nxf = fine_shape
    _, nzc, nyc, nxc = r_coarse.shape
    zi0, zi1, tz = _clamped_linear_coords(nzf, nzc)
    yi0, yi1, ty = _clamped_linear_coords(nyf, nyc)
    xi0, xi1, tx = _clamped_linear_coords(nxf, nxc)
    out = np.zeros((3, nzf, nyf, nxf))
    for c in range(3):
        v = r_coarse[c]
        acc = np.zeros((nzf, nyf, nxf))
        for zi, wz in ((zi0, 1 - tz), (zi1, tz)):
            for yi, wy in ((yi0, 1 - ty), (yi1, ty)):
                for xi, wx in ((xi0, 1 - tx), (xi1, tx)):
                    w = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
                    acc += w * v[np.ix_(zi, yi, xi)]
        out[c] = 2.0 * acc
    return out


# ---------------------------------------------------------------------------
# Sec. 2.1, I_m(x + v(x)); Sec. 2.3 kernel 5 (interpolation kernel)
# Reading R6: trilinear, sample position clamped to [0, n-1] per axis.
# ---------------------------------------------------------------------------

def warp(I_m, r):
    """Deformed moving image I_m^(k)(x) = I_m(x + r(x)) (Sec. 2.1; Sec. 2.3 kernel 5),
    trilinear interpolation with the sample position clamped to the volume (R6)."""
    I_m = np.asarray(I_m, np.float64)
    r = np.asarray(r, np.float64)
    nz, ny, nx = I_m.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    px = np.clip(x + r[0], 0.0, nx - 1)
    py = np.clip(y + r[1], 0.0, ny - 1)
    pz = np.clip(z + r[2], 0.0, nz - 1)
    x0 = np.floor(px).astype(np.int64)
    y0 = np.floor(py).astype(np.int64)
    z0 = np.floor(pz).astype(np.int64)
    tx, ty, tz = px - x0, py - y0, pz - z0
    x1 = np.minimum(x0 + 1, nx - 1)
    y1 = np.minimum(y0 + 1, ny - 1)
    z1 = np.minimum(z0 + 1, nz - 1)
    out = np.zeros(I_m.shape)
    for zi, wz in ((z0, 1 - tz), (z1, tz)):
        for yi, wy in ((y0, 1 - ty), (y1, ty)):
            for xi, wx in ((x0, 1 - tx), (x1, tx)):
                out += wz * wy * wx * I_m[zi, yi, xi]
    return out


def warp_region(I_m, r_region, origin):
    """I_m(x + r(x)) (Sec. 2.1, reading R6) for the voxels x of a sub-box of the grid.

    ``r_region`` is the field on the sub-box ([3][dz][dy][dx]) whose first
    voxel is ``origin`` = (x0, y0, z0) of the full grid of ``I_m``; used to
    evaluate the warp at sampled voxels of large volumes.  Same definition as
    ``warp``: trilinear, sample position clamped to the full grid.
    """
    I_m = np.asarray(I_m, np.float64)
    r = np.asarray(r_region, np.float64)
    nz, ny, nx = I_m.shape
    _, dz, dy, dx = r.shape
    x0, y0, z0 = origin
    z, y, x = np.meshgrid(np.arange(z0, z0 + dz), np.arange(y0, y0 + dy), np.arange(x0, x0 + dx),
                          indexing="ij")
    p = [np.clip(x + r[0], 0.0, nx - 1), np.clip(y + r[1], 0.0, ny - 1), np.clip(z + r[2], 0.0, nz - 1)]
    lo = [np.floor(q).astype(np.int64) for q in p]
    t = [q - i for q, i in zip(p, lo)]
    hi = [np.minimum(i + 1, n - 1) for i, n in zip(lo, (nx, ny, nz))]
    out = np.zeros(r.shape[1:])
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                w = (t[0] if cx else 1 - t[0]) * (t[1] if cy else 1 - t[1]) * (t[2] if cz else 1 - t[2])
                out += w * I_m[(hi if cz else lo)[2], (hi if cy else lo)[1], (hi if cx else lo)[0]]
    return out


# ---------------------------------------------------------------------------
# Eq. (3): raw moments of a patch; reading R7: truncated box at the borders
# ---------------------------------------------------------------------------

def box_sum(X, half):
    """Patch sum of Eq. (3) (truncated box, reading R7): the sum of X over the box
    |dx|<=hx, |dy|<=hy, |dz|<=hz clipped to the volume.

    ``half`` = (hx, hy, hz).  Out-of-volume positions contribute nothing.
    """
    X = np.asarray(X, np.float64)
    out = X
    for comp, h in enumerate(half):
        ax = ARRAY_AXIS[comp]
        n = out.shape[ax]
        acc = np.zeros(out.shape)
        for d in range(-h, h + 1):
            # acc[i] += out[i + d] where 0 <= i + d < n
            lo, hi = max(0, -d), min(n, n - d)
            if lo >= hi:
                continue
            dst = [slice(None)] * 3
            src = [slice(None)] * 3
            dst[ax] = slice(lo, hi)
            src[ax] = slice(lo + d, hi + d)
            acc[tuple(dst)] += out[tuple(src)]
        out = acc
    return out


def box_count(shape, half):
    """n(x) of Eq. (3) for the truncated box (reading R7): the number of in-volume
    voxels of the box around each voxel."""
    return box_sum(np.ones(shape), half)


def patch_moments(X, half):
    """First and second raw moments E(X), E(X^2) of the patch around each voxel (Eq. 3)."""
    n = box_count(X.shape, half)
    E1 = box_sum(X, half) / n
    E2 = box_sum(np.asarray(X, np.float64) ** 2, half) / n
    return E1, E2


def patch_std(E1, E2):
    """STD = sqrt(E(X^2) - E(X)^2) (Appendix, Eq. A.4), clipped at 0 for rounding."""
    return np.sqrt(np.maximum(E2 - E1 * E1, 0.0))


# ---------------------------------------------------------------------------
# Eqs. (2)-(6) and Appendix A.1-A.7: moment matching; Sec. 2.2: I'_s = a I_s + b
# Reading R9: a = 0 where the CBCT patch variance is <= var_floor.
# ---------------------------------------------------------------------------

def intensity_coefficients(m, I_s, half, var_floor=1e-6):
    """Per-voxel a(x), b(x) of Eqs. (5), (6) from patches of I_m^(k) and I_s.

    a = STD(M) / STD(S),  b = E(M) - a E(S).  Where Var(S) <= var_floor the
    ratio is undefined; a = 0 there (so I'_s = E(M)).
    """
    EM, EM2 = patch_moments(m, half)
    ES, ES2 = patch_moments(I_s, half)
    var_m = np.maximum(EM2 - EM * EM, 0.0)
    var_s = np.maximum(ES2 - ES * ES, 0.0)
    std_m = np.where(var_m > var_floor, np.sqrt(var_m), 0.0)
    ok = var_s > var_floor
    std_s = np.sqrt(np.where(ok, var_s, 1.0))
    a = np.where(ok, std_m / std_s, 0.0)
    b = EM - a * ES
    return a, b


def correct(m, I_s, half, var_floor=1e-6):
    """Intensity-corrected static image I'_s = a I_s + b (Sec. 2.2, last paragraph)."""
    a, b = intensity_coefficients(m, I_s, half, var_floor)
    return a * np.asarray(I_s, np.float64) + b


# ---------------------------------------------------------------------------
# Sec. 2.3 kernel 3 (gradient kernel); reading R10: central differences in
# the interior, one-sided first-order differences at the faces, voxel units.
# ---------------------------------------------------------------------------

def gradient(f):
    """Image gradient of Sec. 2.3 kernel 3 (reading R10: central differences inside,
    one-sided at the faces, voxel units), returned as [3][nz][ny][nx], components (x, y, z)."""
    f = np.asarray(f, np.float64)
    g = np.zeros((3,) + f.shape)
    for comp in range(3):
        ax = ARRAY_AXIS[comp]
        n = f.shape[ax]
        if n < 2:
            continue
        fm = np.moveaxis(f, ax, 0)
        gm = np.moveaxis(g[comp], ax, 0)
        gm[1:n - 1] = (fm[2:] - fm[:n - 2]) / 2.0
        gm[0] = fm[1] - fm[0]
        gm[n - 1] = fm[n - 1] - fm[n - 2]
    return g


# ---------------------------------------------------------------------------
# Eq. (1): demons force.  Reading R1: the image difference is taken as
# (I'_s - I_m^(k)) so that adding dr moves I_m(x + r) toward I_s under the
# Sec. 2.1 convention.  Reading R11: a term is 0 where its denominator is
# <= 1e-9.  Reading R2: THIRION = first (passive) term; DOUBLE = both terms.
# ---------------------------------------------------------------------------

def force(m, f, mode=FORCE_THIRION, den_floor=1e-9):
    """Demons force of Eq. (1) (Algorithm A1 step 4; readings R1, R2, R11): the
    displacement increment dr at every voxel ([3][nz][ny][nx])."""
    m = np.asarray(m, np.float64)
    f = np.asarray(f, np.float64)
    diff = f - m
    gf = gradient(f)
    den = (gf ** 2).sum(axis=0) + diff ** 2
    safe = np.where(den > den_floor, den, 1.0)
    dr = np.where(den > den_floor, diff / safe, 0.0) * gf
    if mode == FORCE_DOUBLE:
        gm = gradient(m)
        den2 = (gm ** 2).sum(axis=0) + diff ** 2
        safe2 = np.where(den2 > den_floor, den2, 1.0)
        dr = dr + np.where(den2 > den_floor, diff / safe2, 0.0) * gm
    return dr


# ---------------------------------------------------------------------------
# Algorithm A1 step 6 and Sec. 2.3 kernel 2: Gaussian regularisation of r.
# Reading R12: sampled exp(-i^2 / 2 sigma^2), |i| <= R, separable, weights
# renormalised over the in-volume taps of each axis.
# ---------------------------------------------------------------------------

def gaussian_taps(sigma, radius=0):
    """Algorithm A1 step 6 (reading R12): unnormalised taps w_i = exp(-i^2 / (2 sigma^2)),
    i = -R..R (R = ceil(3 sigma))."""
    if radius <= 0:
        radius = int(math.ceil(3.0 * sigma))
    i = np.arange(-radius, radius + 1, dtype=np.float64)
    return np.exp(-(i * i) / (2.0 * sigma * sigma))


def gaussian_smooth(v, sigma, radius=0):
    """Algorithm A1 step 6 (reading R12): separable Gaussian of a scalar volume,
    renormalised over the in-volume taps of each axis."""
    w = gaussian_taps(sigma, radius)
    R = (len(w) - 1) // 2
    out = np.asarray(v, np.float64)
    for ax in (2, 1, 0):            # x, then y, then z
        n = out.shape[ax]
        num = np.zeros(out.shape)
        den = np.zeros(n)
        for k in range(-R, R + 1):
            lo, hi = max(0, -k), min(n, n - k)
            if lo >= hi:
                continue
            dst = [slice(None)] * 3
            src = [slice(None)] * 3
            dst[ax] = slice(lo, hi)
            src[ax] = slice(lo + k, hi + k)
            num[tuple(dst)] += w[k + R] * out[tuple(src)]
            den[lo:hi] += w[k + R]
        shape = [1, 1, 1]
        shape[ax] = n
        out = num / den.reshape(shape)
    return out


def gaussian_smooth_field(r, sigma, radius=0):
    """Apply the Gaussian to each of the three field components independently."""
    return np.stack([gaussian_smooth(r[c], sigma, radius) for c in range(3)])


# ---------------------------------------------------------------------------
# Sec. 2.3 stopping criterion.  Reading R5: |.| is the per-voxel Euclidean
# norm; l = +inf while sum |r| = 0; stop once k >= window and
# l^(k-window) - l^(k) <= eps.
# ---------------------------------------------------------------------------

def relative_norm(dr, r):
    """Convergence norm of Sec. 2.3 (reading R5): l^(k) = sum |dr^(k+1)| / sum |r^(k)|."""
    num = np.sqrt((np.asarray(dr, np.float64) ** 2).sum(axis=0)).sum()
    den = np.sqrt((np.asarray(r, np.float64) ** 2).sum(axis=0)).sum()
    return math.inf if den == 0.0 else num / den


def should_stop(history, eps, window=10):
    """Stop rule of Sec. 2.3 (reading R5): after at least `window` iterations, stop
    once l^(k - window) - l^(k) <= eps."""
    k = len(history) - 1
    if eps <= 0 or k < window:
        return False
    a, b = history[k - window], history[k]
    if math.isinf(a) or math.isinf(b):
        return False
    return a - b <= eps


# ---------------------------------------------------------------------------
# Algorithm A1: one iteration at one level, and the whole driver
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# Eqs. (7)-(10), Sec. 2.3 and Algorithm A1 step 2: the mask xi of the voxels
# whose a, b (Eqs. 5-6) cannot be trusted, and their interpolation from the
# trusted ones, weighted by CBCT intensity similarity.
# Readings (R17-R20):
#  R17 xi = 1 also where Var(S) <= var_floor, where a is undefined.
#  R18 HU0 = hu0_factor |dHU| with dHU the global shift of Sec. 2.3 (factor 2);
#      a_m is the median of a over the voxels where both patch variances exceed
#      var_floor (a patch where the CT is constant gives a = 0 whatever the
#      CBCT, which says nothing about their intensity scale), at the finest
#      level with r = 0, before the first iteration; a_min = a_lo a_m,
#      a_max = a_hi a_m (0.5 and 1.5).
#  R19 Fill passes are Jacobi sweeps: a pass averages over the neighbours in T
#      that were known before it (xi = 0, or filled by an earlier pass); a
#      voxel without such a neighbour waits for a later pass.  Passes stop when
#      no voxel is left, when a pass fills nothing, or after max_passes; a
#      voxel never filled keeps a = b = 0 (the paper's initial value).
#  R20 The weight exponent (I_s(i) - I_s(x))^2 / h^2 is capped at 80, so that
#      a voxel with a known neighbour always gets a positive weight sum in any
#      floating-point precision (exp(-80) ~ 1.8e-35 is a normal float).
# ---------------------------------------------------------------------------

FILL_EXP_CAP = 80.0


def ratio_median(I_m, I_s, half, var_floor=1e-6):
    """a_m of Sec. 2.3: median of a = STD(M)/STD(S) with r = 0 (m = I_m).

    Over the voxels where Var(M) and Var(S) both exceed var_floor (reading R18)."""
    EM, EM2 = patch_moments(I_m, half)
    ES, ES2 = patch_moments(I_s, half)
    var_m = np.maximum(EM2 - EM * EM, 0.0)
    var_s = np.maximum(ES2 - ES * ES, 0.0)
    ok = (var_s > var_floor) & (var_m > var_floor)
    a = np.sqrt(var_m[ok]) / np.sqrt(var_s[ok])
    return float(np.median(a)) if a.size else 0.0


def mask_xi(m, I_s, a, valid, hu0, a_min, a_max):
    """xi of Eq. (7): 1 where |I_m^(k) - I_s| > HU0 or a is outside
    [a_min, a_max]; also where a is undefined (valid false, reading R17)."""
    m = np.asarray(m, np.float64)
    I_s = np.asarray(I_s, np.float64)
    return (np.abs(m - I_s) > hu0) | (~valid) | (a < a_min) | (a > a_max)


def _shifted(X, d, fill):
    """Helper of the box T of Eqs. (8)-(10): Y[i] = X[i + d] where i + d is inside the
    volume, else `fill`."""
    Y = np.full(X.shape, fill, dtype=X.dtype)
    src, dst = [], []
    for ax, dd in zip((2, 1, 0), d):
        n = X.shape[ax]
        lo, hi = max(0, -dd), min(n, n - dd)
        if lo >= hi:
            return Y
        src.append((ax, slice(lo + dd, hi + dd)))
        dst.append((ax, slice(lo, hi)))
    s_src = [slice(None)] * 3
    s_dst = [slice(None)] * 3
    for (ax, sl_s), (_, sl_d) in zip(src, dst):
        s_src[ax] = sl_s
        s_dst[ax] = sl_d
    Y[tuple(s_dst)] = X[tuple(s_src)]
    return Y


def fill_coefficients(a, b, xi, I_s, h, t_half=(3, 3, 1), max_passes=32):
    """Eqs. (8)-(10): a, b at xi = 1 from the known voxels of the box T.

    T has half sizes t_half = (tx, ty, tz) (7 x 7 x 3 in Sec. 2.3 -> (3, 3, 1)),
    truncated at the volume.  Weights w_i = exp(-(I_s(i) - I_s(x))^2 / h^2)
    (exponent capped, R20).  Jacobi passes (R19).  Returns (a, b, stamp):
    stamp is 0 where xi = 0, the pass that filled the voxel, or -1.
    """
    xi = np.asarray(xi, bool)
    I_s = np.asarray(I_s, np.float64)
    a = np.where(xi, 0.0, np.asarray(a, np.float64))
    b = np.where(xi, 0.0, np.asarray(b, np.float64))
    stamp = np.where(xi, -1, 0).astype(np.int64)
    offsets = [(dx, dy, dz) for dz in range(-t_half[2], t_half[2] + 1)
               for dy in range(-t_half[1], t_half[1] + 1)
               for dx in range(-t_half[0], t_half[0] + 1)]
    for p in range(1, max_passes + 1):
        todo = stamp < 0
        if not todo.any():
            break
        known = (stamp >= 0).astype(np.float64)
        num_a = np.zeros(a.shape)
        num_b = np.zeros(a.shape)
        den = np.zeros(a.shape)
        for d in offsets:
            k = _shifted(known, d, 0.0)
            e = ((_shifted(I_s, d, 0.0) - I_s) / h) ** 2
            w = np.exp(-np.minimum(e, FILL_EXP_CAP)) * k     # Eq. (10), known neighbours only
            num_a += w * _shifted(a, d, 0.0)
            num_b += w * _shifted(b, d, 0.0)
            den += w
        fill = todo & (den > 0.0)
        if not fill.any():
            break
        a[fill] = num_a[fill] / den[fill]                  # Eq. (8)
        b[fill] = num_b[fill] / den[fill]                  # Eq. (9)
        stamp[fill] = p
    return a, b, stamp


@dataclass
class MaskState:
    """Thresholds of Eq. (7) fixed before the first iteration (reading R18)."""
    hu0: float
    a_min: float
    a_max: float


def correct_masked(m, I_s, half, mask: MaskState, h, t_half=(3, 3, 1), max_passes=32,
                   var_floor=1e-6):
    """I'_s = a I_s + b with a, b from Eqs. (5)-(6) where xi = 0 and from the
    fill of Eqs. (8)-(10) where xi = 1 (Algorithm A1 steps 1-3).

    Returns (I'_s, xi, stamp)."""
    EM, EM2 = patch_moments(m, half)
    ES, ES2 = patch_moments(I_s, half)
    var_s = np.maximum(ES2 - ES * ES, 0.0)
    valid = var_s > var_floor
    a, b = intensity_coefficients(m, I_s, half, var_floor)
    xi = mask_xi(m, I_s, a, valid, mask.hu0, mask.a_min, mask.a_max)
    a, b, stamp = fill_coefficients(a, b, xi, I_s, h, t_half, max_passes)
    return a * np.asarray(I_s, np.float64) + b, xi, stamp


@dataclass
class Params:
    patch: tuple = (3, 3, 3)       # odd sizes (px, py, pz); Sec. 3.3 uses 3x3x3
    sigma: float = 1.0             # Gaussian sigma in voxels (not given by the paper)
    radius: int = 0                # 0 -> ceil(3 sigma)
    levels: int = 2                # Sec. 2.3 uses two levels
    iters: List[int] = field(default_factory=lambda: [50, 50])  # coarsest first
    stop_eps: float = 0.0          # 1e-4 in Sec. 2.3; 0 = fixed iteration counts
    stop_window: int = 10
    force_mode: int = FORCE_THIRION
    global_shift: bool = True
    var_floor: float = 1e-6
    den_floor: float = 1e-9
    # Eqs. (7)-(10); mask_mode 0 keeps xi = 0 everywhere
    mask_mode: int = 0
    hu0_factor: float = 2.0        # HU0 = hu0_factor |dHU| (Sec. 2.3)
    a_lo: float = 0.5              # a_min = a_lo a_m
    a_hi: float = 1.5              # a_max = a_hi a_m
    fill_h: float = 50.0           # h of Eq. (10), HU (not given by the paper)
    fill_t: tuple = (7, 7, 3)      # T (Sec. 2.3)
    fill_passes: int = 32
    # reading R4: 0 smooths r + dr (Algorithm A1 step 6); 1 smooths dr and adds it
    # to r (the order of Sec. 2.1)
    smooth_mode: int = 0

    @property
    def half(self):
        return tuple((p - 1) // 2 for p in self.patch)

    @property
    def fill_half(self):
        return tuple((t - 1) // 2 for t in self.fill_t)


def iteration(I_m, I_s, r, p: Params, mask: MaskState = None):
    """One pass of Algorithm A1 steps 1-6 at one level.

    Returns (r_new, dr, l, extras) where extras holds m = I_m^(k) and f = I'_s.
    Step 2 (interpolation of a, b where xi = 1, Eqs. 7-10) runs when
    p.mask_mode is set (thresholds in `mask`); otherwise xi = 0 everywhere.
    """
    m = warp(I_m, r)                                   # update the moving image
    if p.mask_mode:
        f, _xi, _st = correct_masked(m, I_s, p.half, mask, p.fill_h, p.fill_half, p.fill_passes,
                                     p.var_floor)      # steps 1-3
    else:
        f = correct(m, I_s, p.half, p.var_floor)       # steps 1 and 3
    dr = force(m, f, p.force_mode, p.den_floor)        # step 4
    if p.smooth_mode:                                  # Sec. 2.1 order
        r_new = r + gaussian_smooth_field(dr, p.sigma, p.radius)
    else:
        u = r + dr                                     # step 5
        r_new = gaussian_smooth_field(u, p.sigma, p.radius)  # step 6
    l = relative_norm(dr, r)
    return r_new, dr, l, {"m": m, "f": f}


def build_pyramid(img, levels):
    """Sec. 2.3 multi-scale strategy (reading R13): finest level first, each next
    level the 2x2x2 mean of the previous."""
    pyr = [np.asarray(img, np.float64)]
    for _ in range(1, levels):
        pyr.append(downsample2(pyr[-1]))
    return pyr


def register(I_m, I_s, p: Params, return_history=False):
    """Algorithm A1: global shift, pyramid, coarse-to-fine demons with correction.

    Returns the finest-level field r ([3][nz][ny][nx], voxel units) and, with
    ``return_history``, the per-level list of l^(k) values and the corrected
    static image at the last iteration.
    """
    I_m = np.asarray(I_m, np.float64)
    I_s = np.asarray(I_s, np.float64)
    shifted, dhu = global_shift(I_m, I_s)
    if p.global_shift:
        I_s = shifted
    mask = None
    if p.mask_mode:                                     # reading R18
        a_m = ratio_median(I_m, I_s, p.half, p.var_floor)
        mask = MaskState(p.hu0_factor * abs(dhu), p.a_lo * a_m, p.a_hi * a_m)
    pm = build_pyramid(I_m, p.levels)
    ps = build_pyramid(I_s, p.levels)
    r = np.zeros((3,) + pm[-1].shape)
    history = []
    f = None
    for lev in range(p.levels - 1, -1, -1):
        n_it = p.iters[p.levels - 1 - lev]
        hist = []
        for _k in range(n_it):
            r, _dr, l, ex = iteration(pm[lev], ps[lev], r, p, mask)
            f = ex["f"]
            hist.append(l)
            if should_stop(hist, p.stop_eps, p.stop_window):
                break
        history.append(hist)
        if lev > 0:
            r = upsample_field2(r, pm[lev - 1].shape)
    if return_history:
        return r, history, f
    return r


# ---------------------------------------------------------------------------
# Differentiable form (not in the paper): SSD between the warped CT and the
# corrected CBCT, and its adjoint with respect to the field.
# Reading R15: L = sum_x (m(x) - I'_s(x))^2 with m = I_m(x + r(x)) and I'_s
# from Eqs. (5)-(6); the CBCT patch statistics do not depend on r.
# ---------------------------------------------------------------------------

def ssd_loss(I_m, I_s, r, half, var_floor=1e-6):
    """Reading R15 (the differentiable form): L(r) = sum_x (I_m(x + r(x)) - I'_s(x))^2
    with I'_s the moment-matched CBCT of Eqs. (5)-(6)."""
    m = warp(I_m, r)
    f = correct(m, I_s, half, var_floor)
    return float(((m - f) ** 2).sum())


def warp_coord_gradient(I_m, r):
    """d I_m(p) / d p at p = x + r(x) for the trilinear interpolation of Sec. 2.1
    (reading R6), [3][...].

    Zero along an axis where the sample position is clamped to the volume.
    """
    I_m = np.asarray(I_m, np.float64)
    r = np.asarray(r, np.float64)
    nz, ny, nx = I_m.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    raw = [x + r[0], y + r[1], z + r[2]]
    n = [nx, ny, nz]
    lo, t, hi, inside = [], [], [], []
    for a in range(3):
        pa = np.clip(raw[a], 0.0, n[a] - 1)
        i0 = np.floor(pa).astype(np.int64)
        lo.append(i0)
        t.append(pa - i0)
        hi.append(np.minimum(i0 + 1, n[a] - 1))
        inside.append((raw[a] > 0.0) & (raw[a] < n[a] - 1))
    g = np.zeros((3,) + I_m.shape)
    for a in range(3):
        acc = np.zeros(I_m.shape)
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    c = (cx, cy, cz)
                    w = np.ones(I_m.shape)
                    for b in range(3):
                        if b == a:
                            w = w * (1.0 if c[b] else -1.0)
                        else:
                            w = w * (t[b] if c[b] else 1.0 - t[b])
                    idx = [hi[b] if c[b] else lo[b] for b in range(3)]
                    acc += w * I_m[idx[2], idx[1], idx[0]]
        g[a] = np.where(inside[a], acc, 0.0)
    return g


def ssd_grad(I_m, I_s, r, half, var_floor=1e-6):
    """Reading R15: dL/dr by the adjoint of warp -> patch moments (Eq. 3) ->
    correction (Eqs. 5-6) -> SSD.

    f(x) = z_s(x) sigma_m(x) + mu_m(x) with z_s = (I_s - E(S)) / STD(S)
    (algebraically a I_s + b of Eqs. 5-6).  Back-propagation:
      g_f = -2 (m - f);  g_mu = g_f;  g_sigma = g_f z_s
      g_m(y) = 2 (m - f)(y) + sum_{x: y in box(x)} [g_mu(x)/n(x)
               + g_sigma(x) (m(y) - mu(x)) / (n(x) sigma(x))]
      dL/dr(y) = g_m(y) * dI_m/dp at p = y + r(y).
    The sigma term is 0 where Var(M) <= var_floor (sigma_m is held at 0 there).
    """
    m = warp(I_m, r)
    I_s = np.asarray(I_s, np.float64)
    EM, EM2 = patch_moments(m, half)
    ES, ES2 = patch_moments(I_s, half)
    n = box_count(m.shape, half)
    var_m = np.maximum(EM2 - EM * EM, 0.0)
    var_s = np.maximum(ES2 - ES * ES, 0.0)
    ok_m = var_m > var_floor
    ok_s = var_s > var_floor
    sig_m = np.where(ok_m, np.sqrt(np.where(ok_m, var_m, 1.0)), 0.0)
    z_s = np.where(ok_s, (I_s - ES) / np.sqrt(np.where(ok_s, var_s, 1.0)), 0.0)
    f = z_s * sig_m + EM
    g_f = -2.0 * (m - f)
    g_mu = g_f
    g_sig = g_f * z_s
    A = g_mu / n
    B = np.where(ok_m, g_sig / (n * np.where(ok_m, sig_m, 1.0)), 0.0)
    C = B * EM
    g_m = 2.0 * (m - f) + box_sum(A, half) + m * box_sum(B, half) - box_sum(C, half)
    return g_m[None] * warp_coord_gradient(I_m, r)


# ---------------------------------------------------------------------------
# Sec. 2.4.3: evaluation metrics between two images (not on the iteration
# path): normalised mutual information and the RMSE of binary Canny edge
# images, Eq. (11).  Both are written here as their plain definitions in
# float64; the GPU takes the same decisions in float32, so a test accepts a
# different decision only where the float64 margin of that decision is within
# float32 rounding.  Readings:
#  R21 NMI = 2 I(A;B) / (H(A) + H(B)) (it ranges over [0, 1] as the paper says),
#      entropies of a joint histogram with `bins` bins per image over each
#      image's [min, max]; bin(v) = floor((v - min) * bins / (max - min)),
#      clamped to bins - 1; NMI = 1 when both images are constant.
#  R22 Canny edges per transverse slice (2-D): Gaussian smoothing (sigma,
#      taps |i| <= ceil(3 sigma), renormalised over in-slice taps, x then y),
#      central-difference gradient (one-sided at the borders), magnitude
#      M = sqrt(gx^2 + gy^2); non-maximum suppression along the gradient
#      direction quantised to 0, 45, 90, 135 degrees (sector boundaries at
#      tan 22.5 = sqrt(2) - 1 and tan 67.5 = sqrt(2) + 1), neighbours outside
#      the slice count as 0, a pixel is kept when M is above 1e-5 max_slice |I|
#      (a constant slice has only rounding-level gradients in finite
#      precision, which relative thresholds would otherwise turn into edges)
#      and M >= both neighbours; strong where M >= t_high max_slice(M), weak
#      where M >= t_low * that threshold; edges = 8-connected components of the
#      kept strong and weak pixels that contain a strong pixel (hysteresis).
# ---------------------------------------------------------------------------

def nmi_bins(X, bins):
    """Reading R21: histogram bin of every value of X (float64), clamped to bins - 1."""
    X = np.asarray(X, np.float64).ravel()
    mn, mx = X.min(), X.max()
    if mx == mn:
        return np.zeros(X.shape, np.int64)
    t = (X - mn) * bins / (mx - mn)
    return np.minimum(np.floor(t).astype(np.int64), bins - 1)


def nmi(A, B, bins=64):
    """Normalised mutual information of two images (reading R21), float64."""
    ia, ib = nmi_bins(A, bins), nmi_bins(B, bins)
    n = ia.size
    joint = np.zeros((bins, bins))
    np.add.at(joint, (ia, ib), 1.0)
    p = joint / n
    pa, pb = p.sum(1), p.sum(0)

    def ent(q):
        q = q[q > 0]
        return float(-(q * np.log(q)).sum())

    ha, hb, hab = ent(pa), ent(pb), ent(p.ravel())
    if ha + hb == 0.0:
        return 1.0
    return 2.0 * (ha + hb - hab) / (ha + hb)


def _canny_taps(sigma):
    """Reading R22: Gaussian taps of the Canny smoothing, normalised, radius ceil(3 sigma)."""
    R = int(math.ceil(3.0 * sigma))
    i = np.arange(-R, R + 1, dtype=np.float64)
    w = np.exp(-i * i / (2.0 * sigma * sigma))
    return w / w.sum(), R


def _smooth_axis(P, w, R, axis):
    """Reading R22: one separable smoothing pass along `axis`, renormalised over the
    taps that fall inside the slice."""
    n = P.shape[axis]
    acc = np.zeros(P.shape)
    nrm = np.zeros(n)
    for k in range(-R, R + 1):
        lo, hi = max(0, -k), min(n, n - k)
        if lo >= hi:
            continue
        src = [slice(None)] * P.ndim
        dst = [slice(None)] * P.ndim
        src[axis] = slice(lo + k, hi + k)
        dst[axis] = slice(lo, hi)
        acc[tuple(dst)] += w[k + R] * P[tuple(src)]
        nrm[lo:hi] += w[k + R]
    shape = [1] * P.ndim
    shape[axis] = n
    return acc / nrm.reshape(shape)


def _diff_axis(S, axis):
    """Reading R22: central difference along one axis, one-sided at the ends."""
    n = S.shape[axis]
    g = np.zeros(S.shape)
    if n < 2:
        return g
    sl = lambda a, b: tuple(slice(a, b) if ax == axis else slice(None) for ax in range(S.ndim))
    g[sl(1, n - 1)] = 0.5 * (S[sl(2, n)] - S[sl(0, n - 2)])
    g[sl(0, 1)] = S[sl(1, 2)] - S[sl(0, 1)]
    g[sl(n - 1, n)] = S[sl(n - 1, n)] - S[sl(n - 2, n - 1)]
    return g


CANNY_TAN1 = math.sqrt(2.0) - 1.0     # tan 22.5 degrees
CANNY_TAN2 = math.sqrt(2.0) + 1.0     # tan 67.5 degrees
CANNY_SECTORS = ((0, 1), (1, 0), (1, 1), (1, -1))   # (dy, dx) of the first neighbour per sector


def canny_slice(P, sigma=1.0, t_low=0.4, t_high=0.2):
    """The quantities behind the Canny decisions of one slice (reading R22), float64:
    a dict with the smoothed slice S, gradient gx, gy, magnitude M, the sector of
    every pixel (0 horizontal gradient, 1 vertical, 2 and 3 the diagonals with
    gx gy > 0 and <= 0), the neighbour magnitudes n1, n2 of every sector
    ([4][ny][nx]), the floor, the strong threshold hi and the weak one lo."""
    P = np.asarray(P, np.float64)
    w, R = _canny_taps(sigma)
    S = _smooth_axis(_smooth_axis(P, w, R, 1), w, R, 0)
    gx = _diff_axis(S, 1)
    gy = _diff_axis(S, 0)
    M = np.sqrt(gx * gx + gy * gy)
    Mp = np.pad(M, 1)                                    # neighbours outside count as 0

    def nb(dy, dx):
        return Mp[1 + dy:1 + dy + M.shape[0], 1 + dx:1 + dx + M.shape[1]]

    ax, ay = np.abs(gx), np.abs(gy)
    sector = np.where(ay <= CANNY_TAN1 * ax, 0, np.where(ay >= CANNY_TAN2 * ax, 1, np.where(gx * gy > 0, 2, 3)))
    n1 = np.stack([nb(dy, dx) for dy, dx in CANNY_SECTORS])
    n2 = np.stack([nb(-dy, -dx) for dy, dx in CANNY_SECTORS])
    hi = t_high * M.max()
    return dict(S=S, gx=gx, gy=gy, M=M, sector=sector, n1=n1, n2=n2, floor=1e-5 * np.abs(P).max(),
                hi=hi, lo=t_low * hi)


def canny_hysteresis(cand, strong):
    """Reading R22: the 8-connected components of `cand` (2-D bool) that contain a
    pixel of `strong`."""
    from scipy import ndimage
    strong = strong & cand
    if not strong.any():
        return np.zeros(cand.shape, bool)
    lab, _ = ndimage.label(cand, structure=np.ones((3, 3), int))
    good = np.unique(lab[strong])
    return np.isin(lab, good[good > 0])


def canny(img, sigma=1.0, t_low=0.4, t_high=0.2):
    """Binary Canny edge image, slice by slice (reading R22); bool [nz][ny][nx]."""
    img = np.asarray(img, np.float64)
    edges = np.zeros(img.shape, bool)
    for z in range(img.shape[0]):
        q = canny_slice(img[z], sigma, t_low, t_high)
        M, sec = q["M"], q["sector"]
        n1 = np.take_along_axis(q["n1"], sec[None], 0)[0]
        n2 = np.take_along_axis(q["n2"], sec[None], 0)[0]
        keep = (M > q["floor"]) & (M >= n1) & (M >= n2)
        edges[z] = canny_hysteresis(keep & (M >= q["lo"]), keep & (M >= q["hi"]))
    return edges


def edge_rmse(E1, E2):
    """Eq. (11): sqrt(sum_i (E1(i) - E2(i))^2 / N) of two binary edge images."""
    E1 = np.asarray(E1, bool)
    E2 = np.asarray(E2, bool)
    return math.sqrt(np.count_nonzero(E1 != E2) / E1.size)
