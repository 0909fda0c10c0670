"""Z-slab decomposition of one registration: the volume is split along z into
slabs, each registered by its own context on its interior planes plus a halo,
with the field's halo planes refreshed from their owners after every
iteration -- the decomposition a multi-device run of one large volume uses,
driven here as independent contexts on one device (device-to-device copies
stand in for the halo messages).

Why a halo of ``R + p_z + d + 3`` planes makes every interior plane exact,
following one iteration of Algorithm A1 backwards from r^(k+1) at plane z:

* the Gaussian (step 6) reads u = r + dr on planes z - R .. z + R;
* dr (Eq. 1, step 4) at a plane z' reads f = I'_s and its central difference,
  so planes z' - 1 .. z' + 1 (the double force also reads m there);
* f (Eqs. 5-6, step 3) at a plane z'' reads the patch moments of m and of I_s
  over z'' - p_z .. z'' + p_z;
* m = I_m(x + r(x)) at a plane z''' reads r there and I_m between
  floor(z''' + r_z) and that plus one, inside z''' - d - 1 .. z''' + d + 1 when
  |r_z| <= d, and a sample is clamped at the buffer's last plane.

So r and m are needed on z +- (R + 1 + p_z) and I_m on z +- (R + p_z + d + 3);
the static image's moments stay inside the same reach.  Planes nearer a
buffer's cut than that come out wrong (truncated patches, renormalised
Gaussian taps, clamped samples) and are overwritten by the next exchange; at
the volume's own faces the buffer ends where the volume does, so the
truncations are the whole volume's.  The global intensity shift and the
fixed-point scales are taken from the whole volume (``quant_max``), which
makes every interior voxel of every slab bit-identical to the whole-volume
run.  Scope: one pyramid level, fixed iteration counts (the convergence
norm's sums are per slab) and the mask off (its median a_m is a whole-volume
statistic).
"""
from __future__ import annotations

import math

from . import disc


def halo_planes(patch, sigma, radius=0, max_disp_z=8.0):
    """Halo depth (planes per side) that keeps a slab's interior exact while
    |r_z| <= max_disp_z voxels (see the module docstring)."""
    R = int(radius) if radius > 0 else int(math.ceil(3.0 * float(sigma)))
    pz = (int(patch[2]) - 1) // 2
    return R + pz + int(math.ceil(float(max_disp_z))) + 3


def slab_plan(nz, nslabs, halo):
    """[(z0, z1, b0, b1)]: interior planes [z0, z1) and buffer planes [b0, b1)
    of each slab; interiors tile [0, nz) in order, as equal as possible."""
    if nslabs < 1 or nz < nslabs:
        raise ValueError("need 1 <= nslabs <= nz")
    if halo < 0:
        raise ValueError("halo must be >= 0")
    base, extra = divmod(nz, nslabs)
    plan, z0 = [], 0
    for s in range(nslabs):
        z1 = z0 + base + (1 if s < extra else 0)
        plan.append((z0, z1, max(0, z0 - halo), min(nz, z1 + halo)))
        z0 = z1
    return plan


def exchange_sources(plan, s):
    """Copies that refill slab s's buffer: [(t, lo, hi)] -- planes [lo, hi) of
    the volume taken from slab t's interior, covering s's buffer in order."""
    _, _, b0, b1 = plan[s]
    out = []
    for t, (z0, z1, _, _) in enumerate(plan):
        lo, hi = max(b0, z0), min(b1, z1)
        if lo < hi:
            out.append((t, lo, hi))
    return out


class SlabRegistration:
    """One volume registered as ``nslabs`` z slabs (one level, fixed counts).

    ``max_disp_z`` bounds |r_z| (voxels) over the run; ``halo`` overrides the
    depth derived from it.  Images are float32 [nz][ny][nx] torch CUDA tensors.
    """

    def __init__(self, nslabs=2, max_disp_z=8.0, halo=None, **kw):
        import torch
        self._torch = torch
        kw = dict(kw)
        if kw.get("levels", 1) != 1:
            raise ValueError("the slab decomposition runs one pyramid level")
        if kw.get("mask_mode", 0) or kw.get("stop_eps", 0.0) > 0.0:
            raise ValueError("the slab decomposition runs with the mask off and fixed counts")
        kw["levels"] = 1
        kw["iters"] = (1 << 30,)                 # counts are driven here
        self.shift = bool(kw.pop("global_shift", True))
        self.kw = kw
        self.nslabs = int(nslabs)
        self.halo = int(halo) if halo is not None else halo_planes(kw.get("patch", (3, 3, 3)), kw.get("sigma", 1.0),
                                                                    kw.get("radius", 0), max_disp_z)
        self.regs = []
        self.plan = None
        self.dims = None

    def close(self):
        for r in self.regs:
            r.close()
        self.regs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_images(self, ct, cbct):
        torch = self._torch
        nz, ny, nx = ct.shape
        is_shift = cbct
        if self.shift:                           # Sec. 2.3: shift I_s by mean(I_m) - mean(I_s), whole volume
            is_shift = torch.empty_like(cbct)
            disc.k_global_shift(ct, cbct, is_shift)
        mx = torch.empty(2, dtype=torch.float32, device=ct.device)
        disc.k_max_abs(ct, mx[0:1])
        disc.k_max_abs(is_shift, mx[1:2])
        qmax = [float(v) for v in mx.cpu()]
        self.close()
        self.plan = slab_plan(nz, self.nslabs, self.halo)
        for (_, _, b0, b1) in self.plan:
            p = disc.make_params(global_shift=False, quant_max=qmax, **self.kw)
            reg = disc.Registration(p)
            reg.set_images(ct[b0:b1].contiguous(), is_shift[b0:b1].contiguous())
            self.regs.append(reg)
        self.dims = (nx, ny, nz)

    def _fields(self):
        torch = self._torch
        nx, ny, _ = self.dims
        out = []
        for reg, (_, _, b0, b1) in zip(self.regs, self.plan):
            f = torch.empty((3, b1 - b0, ny, nx), dtype=torch.float32, device="cuda")
            reg.get_field(f)
            out.append(f)
        return out

    def exchange(self):
        """Refill every slab's buffer field from the owners of its planes."""
        torch = self._torch
        fields = self._fields()
        for s, reg in enumerate(self.regs):
            _, _, b0, b1 = self.plan[s]
            buf = torch.empty_like(fields[s])
            for t, lo, hi in exchange_sources(self.plan, s):
                tb0 = self.plan[t][2]
                buf[:, lo - b0:hi - b0] = fields[t][:, lo - tb0:hi - tb0]
            reg.set_field(0, buf)

    def iterate(self, n):
        for _ in range(int(n)):
            for reg in self.regs:
                reg.iterate(1, sync=False)
            self.exchange()

    def get_field(self):
        """The assembled field [3][nz][ny][nx] (device tensor): each slab's interior."""
        torch = self._torch
        nx, ny, nz = self.dims
        out = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
        for f, (z0, z1, b0, _) in zip(self._fields(), self.plan):
            out[:, z0:z1] = f[:, z0 - b0:z1 - b0]
        return out
