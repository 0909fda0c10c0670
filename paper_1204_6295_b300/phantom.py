"""Seeded synthetic CT / CBCT pairs for the DISC registration workloads.

This module only draws inputs. It holds none of the registration arithmetic:
there is no interpolation, no patch statistic, no force and no filter here.
The CBCT is produced by evaluating the *analytic* phantom at displaced
coordinates ``x + u(x)`` (so that ``CT(x + u(x)) = CBCT_primary(x)``, the
relation of Sec. 2.1), then adding the artifacts that motivate the method
(Sec. 1 and Sec. 2.4.1: cupping from scatter, streaks, noise).

Both the oracle-based tests and the CUDA path are fed the same arrays.

Array layout: C-order ``[nz][ny][nx]`` (x fastest), float32 outputs, built in
float64.  Displacements are in voxel units of the generated grid, stored as
``[3][nz][ny][nx]`` with components (x, y, z).

Workloads (stand-ins for the MC-simulated and clinical head-and-neck data of
Sec. 2.4.1 and Sec. 2.4.2, which are not available):

* ``ellipsoid_pair``: nested ellipsoids (-1000 / 0 / 40 / 1000 HU), a
  sinusoidal field of amplitude 3 voxels and period 32 voxels, radial cupping
  of up to -150 HU and Gaussian noise with sigma 20 HU.
* ``head_neck_pair``: a head-sized anatomy (ellipsoidal skull shell at +1000
  HU, soft tissue split into piecewise-constant regions drawn from U[0, 60]
  HU, air cavities at -1000 HU); a smooth random field of max 8 mm at
  1x1x2 mm voxels; cupping up to -200 HU; a radial streak pattern; noise
  sigma 30 HU.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

SEED_BASE = 12046295


@dataclass
class Pair:
    """One synthetic CT (moving) / CBCT (static) pair and its ground truth."""

    ct: np.ndarray          # [nz][ny][nx] float32, moving image I_m
    cbct: np.ndarray        # [nz][ny][nx] float32, static image I_s
    u_true: np.ndarray      # [3][nz][ny][nx] float32, I_m(x + u) = primary CBCT
    cbct_primary: np.ndarray  # [nz][ny][nx] float32, artifact-free CBCT

    @property
    def shape(self):
        return self.ct.shape

    @property
    def dims(self):
        nz, ny, nx = self.ct.shape
        return nx, ny, nz


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def _smooth_inside(s, width):
    """Soft indicator of ``s < 1`` for a normalised radius ``s``.

    ``width`` is the transition width in units of ``s``; a width of about one
    voxel gives partial-volume-like edges instead of a hard step.
    """
    return np.clip((1.0 - s) / width + 0.5, 0.0, 1.0)


# --------------------------------------------------------------------------
# Config "ellipsoids": 64x64x32 nested ellipsoids
# --------------------------------------------------------------------------

def _ellipsoid_ct(x, y, z, nx, ny, nz):
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    img = np.full(x.shape, -1000.0)
    levels = ((0.45, 0.0), (0.30, 40.0), (0.15, 1000.0))
    prev = -1000.0
    for frac, hu in levels:
        a, b, c = frac * nx, frac * ny, frac * nz
        s = np.sqrt(((x - cx) / a) ** 2 + ((y - cy) / b) ** 2 + ((z - cz) / c) ** 2)
        width = 1.0 / min(a, b, c)
        ins = _smooth_inside(s, width)
        img = img + ins * (hu - prev)
        prev = hu
    return img


def ellipsoid_pair(nx=64, ny=64, nz=32, seed=SEED_BASE + 1, amplitude=3.0,
                   period=32.0, cupping=150.0, noise=20.0):
    """Nested-ellipsoid CT and a deformed, cupped, noisy CBCT."""
    rng = np.random.default_rng(seed)
    x, y, z = _grid(nx, ny, nz)
    w = 2.0 * math.pi / period
    ux = amplitude * np.sin(w * y)
    uy = amplitude * np.sin(w * z)
    uz = amplitude * np.sin(w * x)
    ct = _ellipsoid_ct(x, y, z, nx, ny, nz)
    primary = _ellipsoid_ct(x + ux, y + uy, z + uz, nx, ny, nz)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    rho2 = (x - cx) ** 2 + (y - cy) ** 2
    rho2_max = (max(nx, ny) / 2.0) ** 2
    bias = -cupping * np.clip(1.0 - rho2 / rho2_max, 0.0, None)
    cbct = primary + bias + rng.normal(0.0, noise, size=x.shape)
    u = np.stack([ux, uy, uz])
    return Pair(ct.astype(np.float32), cbct.astype(np.float32),
                u.astype(np.float32), primary.astype(np.float32))


# --------------------------------------------------------------------------
# Config "head and neck": skull shell, soft-tissue regions, air cavities
# --------------------------------------------------------------------------

class _HeadAnatomy:
    """Analytic head phantom, evaluated at arbitrary (possibly displaced) points."""

    def __init__(self, rng, nx, ny, nz, spacing):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.c = np.array([(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0])
        sx, sy, sz = spacing
        # physical semi-axes (mm) scaled to the grid's field of view
        fov = np.array([nx * sx, ny * sy, nz * sz])
        self.spacing = np.array(spacing, dtype=np.float64)
        self.outer = fov * np.array([0.42, 0.46, 0.44])       # skull outer surface
        self.inner = self.outer - np.array([7.0, 7.0, 7.0])   # 7 mm bone
        self.body = fov * np.array([0.47, 0.49, 0.48])        # skin surface
        n_seeds = 16
        self.seeds = (rng.uniform(-0.8, 0.8, size=(n_seeds, 3)) * self.inner)
        self.seed_hu = rng.uniform(0.0, 60.0, size=n_seeds)
        n_cav = 4
        self.cav_c = rng.uniform(-0.5, 0.5, size=(n_cav, 3)) * self.inner
        self.cav_r = rng.uniform(0.08, 0.16, size=(n_cav, 1)) * self.inner.min() * np.array(
            [[1.0, 1.0, 0.8]])
        self.body_hu = 30.0

    def __call__(self, x, y, z):
        # displacement from the centre in mm
        px = (x - self.c[0]) * self.spacing[0]
        py = (y - self.c[1]) * self.spacing[1]
        pz = (z - self.c[2]) * self.spacing[2]
        edge_mm = 1.0
        img = np.full(x.shape, -1000.0)

        def radius(axes):
            return np.sqrt((px / axes[0]) ** 2 + (py / axes[1]) ** 2 + (pz / axes[2]) ** 2)

        s_body = radius(self.body)
        in_body = _smooth_inside(s_body, edge_mm / self.body.min())
        # soft tissue: piecewise-constant regions (nearest seed)
        d = ((px[None] - self.seeds[:, 0, None, None, None]) ** 2
             + (py[None] - self.seeds[:, 1, None, None, None]) ** 2
             + (pz[None] - self.seeds[:, 2, None, None, None]) ** 2)
        tissue = self.seed_hu[np.argmin(d, axis=0)]
        del d
        s_in = radius(self.inner)
        inside_skull = _smooth_inside(s_in, edge_mm / self.inner.min())
        soft = self.body_hu * (1.0 - inside_skull) + tissue * inside_skull
        img = img + in_body * (soft + 1000.0)
        # bone shell between the inner and outer skull surfaces
        s_out = radius(self.outer)
        shell = _smooth_inside(s_out, edge_mm / self.outer.min()) * (1.0 - inside_skull)
        img = img + shell * (1000.0 - soft)
        # air cavities
        for k in range(self.cav_c.shape[0]):
            r = self.cav_r[k]
            s = np.sqrt(((px - self.cav_c[k, 0]) / r[0]) ** 2 + ((py - self.cav_c[k, 1]) / r[1]) ** 2
                        + ((pz - self.cav_c[k, 2]) / r[2]) ** 2)
            cav = _smooth_inside(s, edge_mm / r.min())
            img = img + cav * (-1000.0 - img)
        return img


def _draw_modes(rng, n_modes=6):
    """Random low-frequency sinusoid modes for the three field components."""
    modes = []
    for _ in range(3):
        k = rng.uniform(0.5, 2.0, size=(n_modes, 3)) * rng.choice([-1.0, 1.0], size=(n_modes, 3))
        ph = rng.uniform(0, 2 * math.pi, size=n_modes)
        amp = rng.uniform(0.5, 1.0, size=n_modes)
        modes.append((k, ph, amp))
    return modes


def _eval_modes(modes, x, y, z, dims):
    """Raw (unscaled) field components at the grid points of a z-slab.

    ``x, y, z`` are the meshgrid coordinates of the slab (only their 1-D axes
    are used): each mode sin(2 pi (kx x/nx + ky y/ny + kz z/nz) + ph) is the
    imaginary part of a product of three 1-D complex exponentials.
    """
    nx, ny, nz = dims
    xs, ys, zs = x[0, 0, :], y[0, :, 0], z[:, 0, 0]
    out = []
    for k, ph, amp in modes:
        acc = np.zeros(x.shape)
        for i in range(k.shape[0]):
            ex = np.exp(2j * math.pi * k[i, 0] * xs / nx)
            ey = np.exp(2j * math.pi * k[i, 1] * ys / ny)
            ez = np.exp(2j * math.pi * k[i, 2] * zs / nz) * (amp[i] * np.exp(1j * ph[i]))
            acc += (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).imag
        out.append(acc)
    return out


def head_neck_pair(nx=256, ny=256, nz=128, seed=SEED_BASE + 2, spacing=(1.0, 1.0, 2.0),
                   max_mm=8.0, cupping=200.0, streak=40.0, noise=30.0):
    """Head-and-neck-sized CT / CBCT pair (Sec. 2.4.2 sizes), seed-fixed.

    The field is a sum of random sinusoids scaled so that its peak physical
    magnitude is ``max_mm`` (8 voxels in x/y and 4 in z at 1x1x2 mm).
    """
    rng = np.random.default_rng(seed)
    anatomy = _HeadAnatomy(rng, nx, ny, nz, spacing)
    modes = _draw_modes(np.random.default_rng(seed + 7919))
    noise_rng = np.random.default_rng(seed + 104729)
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    rho_max = math.hypot(cx, cy)
    n_streaks = 5
    theta_j = rng.uniform(0, 2 * math.pi, size=n_streaks)
    k_j = rng.integers(3, 7, size=n_streaks)
    slab = max(1, (1 << 21) // (nx * ny))
    sp = np.asarray(spacing, dtype=np.float64)
    starts = list(range(0, nz, slab))
    # the slabs are independent numpy work (which releases the GIL): threads
    from concurrent.futures import ThreadPoolExecutor
    workers = max(1, min(len(starts), os.cpu_count() or 1))

    # pass 1: peak physical magnitude of the raw field over the whole grid
    def slab_peak(zs):
        x, y, z = _grid(nx, ny, min(nz, zs + slab) - zs)
        c = _eval_modes(modes, x, y, z + zs, (nx, ny, nz))
        return float(np.sqrt((c[0] * sp[0]) ** 2 + (c[1] * sp[1]) ** 2 + (c[2] * sp[2]) ** 2).max())

    with ThreadPoolExecutor(max_workers=workers) as ex:
        peak = max([0.0] + list(ex.map(slab_peak, starts)))
    # field in mm = raw * sp * (max_mm / peak); in voxels divide by sp again
    scale = max_mm / peak
    ct = np.empty((nz, ny, nx), np.float32)
    cbct = np.empty((nz, ny, nx), np.float32)
    prim = np.empty((nz, ny, nx), np.float32)
    u = np.empty((3, nz, ny, nx), np.float32)
    base = np.empty((nz, ny, nx), np.float64)     # the CBCT before its noise

    def slab_images(zs):
        ze = min(nz, zs + slab)
        x, y, z = _grid(nx, ny, ze - zs)
        z = z + zs
        c = _eval_modes(modes, x, y, z, (nx, ny, nz))
        ux, uy, uz = c[0] * scale, c[1] * scale, c[2] * scale
        ct[zs:ze] = anatomy(x, y, z)
        p = anatomy(x + ux, y + uy, z + uz)
        prim[zs:ze] = p
        rho = np.hypot(x - cx, y - cy)
        theta = np.arctan2(y - cy, x - cx)
        bias = -cupping * np.clip(1.0 - (rho / rho_max) ** 2, 0.0, None)
        st = np.zeros_like(rho)
        for j in range(n_streaks):
            st += np.cos(k_j[j] * (theta - theta_j[j]))
        st *= streak * np.exp(-rho / (0.35 * rho_max)) / n_streaks
        base[zs:ze] = p + bias + st
        u[0, zs:ze], u[1, zs:ze], u[2, zs:ze] = ux, uy, uz

    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(slab_images, starts))
    # the noise is drawn slab after slab from one generator, in z order
    for zs in starts:
        ze = min(nz, zs + slab)
        cbct[zs:ze] = base[zs:ze] + noise_rng.normal(0.0, noise, size=base[zs:ze].shape)
    return Pair(ct, cbct, u, prim)


def batch_sizes(n_pairs=16, seed=SEED_BASE + 4, choices=(64, 80, 96, 112, 128, 144, 160)):
    """Uneven pair dims (2s, 2s, s) for the batched workload, s drawn per pair."""
    rng = np.random.default_rng(seed)
    s = rng.choice(np.array(choices), size=n_pairs)
    return [(int(2 * v), int(2 * v), int(v)) for v in s]


def _batch_pair_images(args):
    i, (nx, ny, nz), seed = args
    p = head_neck_pair(nx, ny, nz, seed=seed + 1000 * (i + 1))
    return p.ct, p.cbct


def batch_pair_images(n_pairs=16, seed=SEED_BASE + 4, workers=None, indices=None, sizes=None):
    """(CT, CBCT) of the batched workload's pairs, drawn in parallel processes.

    n_pairs head-and-neck pairs of uneven size (2s, 2s, s), s from 64 to 160,
    or of the given (nx, ny, nz) `sizes`; with `indices`, only those pairs (a
    rank's share), in that order.  The worker processes are started with
    'spawn' (safe after CUDA is initialised).
    """
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    if sizes is None:
        sizes = batch_sizes(n_pairs, seed)
    elif len(sizes) != n_pairs:
        raise ValueError("one size per pair")
    if indices is None:
        indices = range(n_pairs)
    jobs = [(i, sizes[i], seed) for i in indices]
    if not jobs:
        return []
    if workers is None:
        workers = max(1, min(len(jobs), os.cpu_count() or 1))
    if workers == 1:
        return [_batch_pair_images(j) for j in jobs]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batch_pair_images, jobs))


def random_volume(shape, seed, lo=-1000.0, hi=1000.0):
    """Uniform random volume (float32) for kernel-level tests."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def random_field(shape, seed, amp=2.0):
    """Uniform random displacement field [3][*shape] (float32), voxel units."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, size=(3,) + tuple(shape)).astype(np.float32)


def smooth_random_field(shape, seed, amp=3.0):
    """Smooth displacement field [3][*shape] from random sinusoids, voxel units."""
    nz, ny, nx = shape
    x, y, z = _grid(nx, ny, nz)
    c = _eval_modes(_draw_modes(np.random.default_rng(seed), n_modes=3), x, y, z, (nx, ny, nz))
    mag = np.sqrt(c[0] ** 2 + c[1] ** 2 + c[2] ** 2).max()
    return (np.stack(c) * (amp / mag)).astype(np.float32)
