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
run.

Pyramid levels: level l halves the grid l times (2 x 2 x 2 means), so slab
cuts and buffer starts sit on multiples of 2^(L-1) planes and a slab's coarse
planes are the whole volume's; the halo must cover the reach at every level,
2^l (R + p_z + ceil(d / 2^l) + 3) fine planes at level l.  At a level's end
every slab up-samples its own buffer (the fine planes of its interior read
coarse planes at most one away) and the fine level starts with an exchange.

The convergence norm l^(k) = sum |dr| / sum |r| (Sec. 2.3) is a ratio of two
whole-volume sums: each slab sums its interior only (``norm_planes``), the two
sums are added over the slabs (the allreduce of a multi-device run) and the
stop rule is applied to the ratio, ending the level in every slab at once.

With one rank per slab, ``halo_exchange`` and ``allreduce_norm_sums`` are the
two collectives of an iteration (point-to-point halo planes, a two-scalar
allreduce) over torch.distributed.
Scope: the mask off (its median a_m is a whole-volume statistic).
"""
from __future__ import annotations

import math

import numpy as np

from . import disc


def halo_planes(patch, sigma, radius=0, max_disp_z=8.0, levels=1):
    """Halo depth (fine planes per side, a multiple of 2^(levels-1)) that keeps
    a slab's interior exact at every level while |r_z| <= max_disp_z fine
    voxels (see the module docstring)."""
    R = int(radius) if radius > 0 else int(math.ceil(3.0 * float(sigma)))
    pz = (int(patch[2]) - 1) // 2
    h = max((1 << l) * (R + pz + int(math.ceil(float(max_disp_z) / (1 << l))) + 3) for l in range(levels))
    align = 1 << (levels - 1)
    return (h + align - 1) // align * align


def slab_plan(nz, nslabs, halo, align=1):
    """[(z0, z1, b0, b1)]: interior planes [z0, z1) and buffer planes [b0, b1)
    of each slab; interiors tile [0, nz) in order, as equal as possible in
    units of `align` planes, and every cut and buffer start is a multiple of
    `align` (halo must be one)."""
    if align < 1 or halo % align:
        raise ValueError("align >= 1 and halo a multiple of it")
    units = (nz + align - 1) // align
    if nslabs < 1 or units < nslabs:
        raise ValueError("need 1 <= nslabs <= ceil(nz / align)")
    if halo < 0:
        raise ValueError("halo must be >= 0")
    base, extra = divmod(units, nslabs)
    plan, u0 = [], 0
    for s in range(nslabs):
        u1 = u0 + base + (1 if s < extra else 0)
        z0, z1 = u0 * align, min(nz, u1 * align)
        plan.append((z0, z1, max(0, z0 - halo), min(nz, z1 + halo)))
        u0 = u1
    return plan


def level_plan(plan, nz, level):
    """The plan in the planes of pyramid level `level` (cuts halved `level` times)."""
    def down(z):
        for _ in range(level):
            z = (z + 1) // 2
        return z
    return [(down(z0), down(z1), down(b0), down(b1)) for z0, z1, b0, b1 in plan]


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


def halo_exchange(plan, rank, buf, dist, group=None):
    """One halo exchange of a multi-rank slab split, rank `rank` owning slab
    `rank` of `plan`: `buf` ([3][b1 - b0][ny][nx] torch tensor, the rank's
    buffer field) gets every plane it holds but does not own from that plane's
    owner, and sends the planes of its interior that other buffers hold.
    Point-to-point messages (one per neighbouring pair and direction, matched by
    the plan that every rank computes alone); `dist` is torch.distributed with an
    initialised process group (NCCL for device tensors, gloo for host ones)."""
    _, _, b0, _ = plan[rank]
    reqs, recvs = [], []
    for s in range(len(plan)):
        if s == rank:
            continue
        for t, lo, hi in exchange_sources(plan, s):
            if t == rank:                          # planes [lo, hi) of my interior, for s
                reqs.append(dist.isend(buf[:, lo - b0:hi - b0].contiguous(), dst=s, group=group))
    for t, lo, hi in exchange_sources(plan, rank):
        if t != rank:                              # planes [lo, hi) of my buffer, from t
            tmp = buf.new_empty((buf.shape[0], hi - lo) + tuple(buf.shape[2:]))
            reqs.append(dist.irecv(tmp, src=t, group=group))
            recvs.append((tmp, lo))
    for q in reqs:
        q.wait()
    for tmp, lo in recvs:
        buf[:, lo - b0:lo - b0 + tmp.shape[1]] = tmp
    return buf


def allreduce_norm_sums(sums, dist, group=None):
    """The two sums behind l^(k) (sum |dr|, sum |r| over a rank's interior planes,
    a float64 tensor of 2) added over the ranks in place: the scalar allreduce of
    the convergence norm (Sec. 2.3)."""
    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums


class SlabRegistration:
    """One volume registered as ``nslabs`` z slabs (fixed counts, mask off).

    ``levels`` and ``iters`` (coarsest first) give the schedule, as for
    Registration; ``max_disp_z`` bounds |r_z| (fine voxels) over the run and
    ``halo`` overrides the depth derived from it.  Images are float32
    [nz][ny][nx] torch CUDA tensors.
    """

    def __init__(self, nslabs=2, max_disp_z=8.0, halo=None, levels=1, iters=(50,), **kw):
        import torch
        self._torch = torch
        kw = dict(kw)
        if kw.get("mask_mode", 0):
            raise ValueError("the slab decomposition runs with the mask off")
        if len(iters) != levels:
            raise ValueError("one iteration count per level (coarsest first)")
        self.levels = int(levels)
        self.iters = [int(n) for n in iters]
        # the stop rule is applied here, to the slabs' summed norms
        self.stop_eps = float(kw.pop("stop_eps", 0.0))
        self.stop_window = int(kw.get("stop_window", 10))
        kw["levels"] = self.levels
        kw["iters"] = tuple(max(1, n) for n in self.iters)   # each exchange restarts a context's count
        self.hist = [[] for _ in range(self.levels)]
        self.shift = bool(kw.pop("global_shift", True))
        self.kw = kw
        self.nslabs = int(nslabs)
        self.align = 1 << (self.levels - 1)
        self.halo = int(halo) if halo is not None else halo_planes(
            kw.get("patch", (3, 3, 3)), kw.get("sigma", 1.0), kw.get("radius", 0), max_disp_z, self.levels)
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
        self.plan = slab_plan(nz, self.nslabs, self.halo, self.align)
        self.hist = [[] for _ in range(self.levels)]
        for (z0, z1, b0, b1) in self.plan:
            p = disc.make_params(global_shift=False, quant_max=qmax, norm_planes=(z0 - b0, z1 - b0), **self.kw)
            reg = disc.Registration(p)
            reg.set_images(ct[b0:b1].contiguous(), is_shift[b0:b1].contiguous())
            self.regs.append(reg)
        self.dims = (nx, ny, nz)

    def _level_dims(self, level):
        nx, ny, _ = self.dims
        for _ in range(level):
            nx, ny = (nx + 1) // 2, (ny + 1) // 2
        return nx, ny

    def _fields(self, level):
        """Each slab's field at `level`."""
        torch = self._torch
        nx, ny = self._level_dims(level)
        out = []
        for reg, (_, _, b0, b1) in zip(self.regs, level_plan(self.plan, self.dims[2], level)):
            f = torch.empty((3, b1 - b0, ny, nx), dtype=torch.float32, device="cuda")
            reg.get_level_field(level, f)
            out.append(f)
        return out

    def exchange(self, level, fields=None):
        """Refill every slab's buffer field at `level` from the owners of its
        planes (fields: the slabs' fields at that level, else read back)."""
        torch = self._torch
        if fields is None:
            fields = self._fields(level)
        plan = level_plan(self.plan, self.dims[2], level)
        for s, reg in enumerate(self.regs):
            _, _, b0, b1 = plan[s]
            buf = torch.empty_like(fields[s])
            for t, lo, hi in exchange_sources(plan, s):
                tb0 = plan[t][2]
                buf[:, lo - b0:hi - b0] = fields[t][:, lo - tb0:hi - tb0]
            reg.set_field(level, buf)

    def _norm_step(self, level):
        """The slabs' interior sums of the iteration just run, added (the allreduce of
        a multi-rank run); True when the stop rule of Sec. 2.3 ends the level
        (disc_norm_stop_rule on the summed history)."""
        sdr = sr = 0.0
        for reg in self.regs:
            s = reg.norm_sums(level, cap=1)      # each exchange restarts the count: this iteration's sums
            sdr += float(s[0, 0])
            sr += float(s[0, 1])
        self.hist[level].append((sdr, sr))
        _, stop = disc.norm_stop_rule(self.hist[level], self.stop_window, self.stop_eps)
        return stop

    def norm_history(self, level):
        """l^(k) of the iterations run at `level` (float32, as a context reports it)."""
        if not self.hist[level]:
            return np.zeros(0, np.float32)
        return disc.norm_stop_rule(self.hist[level], self.stop_window, self.stop_eps)[0]

    def iterate(self):
        """The whole schedule, coarsest level first; returns the iterations run."""
        torch = self._torch
        done = 0
        for level in range(self.levels - 1, -1, -1):
            for _ in range(self.iters[self.levels - 1 - level]):
                for reg in self.regs:
                    reg.iterate(1, sync=False)
                done += 1
                stop = self._norm_step(level)
                self.exchange(level)
                if stop:
                    break
            if level > 0:                        # Algorithm A1: up-sample to the next finer level
                nx, ny = self._level_dims(level - 1)
                fine = []
                for f, (_, _, b0, b1) in zip(self._fields(level), level_plan(self.plan, self.dims[2], level - 1)):
                    rf = torch.empty((3, b1 - b0, ny, nx), dtype=torch.float32, device="cuda")
                    disc.k_upsample_field2(f, rf)
                    fine.append(rf)
                self.exchange(level - 1, fine)
        return done

    def get_field(self):
        """The assembled finest-level field [3][nz][ny][nx] (device tensor): each slab's interior."""
        torch = self._torch
        nx, ny, nz = self.dims
        out = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
        for f, (z0, z1, b0, _) in zip(self._fields(0), self.plan):
            out[:, z0:z1] = f[:, z0 - b0:z1 - b0]
        return out


# ---------------------------------------------------------------------------
# One slab per rank
# ---------------------------------------------------------------------------

class LibdiscSlab:
    """The per-rank engine of run_slab_rank: one registration context on this
    rank's device, over the buffer planes [b0, b1) of its slab.

    ``ct`` and ``cbct_shifted`` are the rank's buffer planes of the CT and of the
    globally shifted CBCT (torch CUDA tensors on the rank's device); ``qmax`` the
    whole volume's largest |I_m| and |I_s| (after the shift), so that every
    interior voxel is computed from the same integers as in a whole-volume run;
    ``norm_planes`` the interior planes relative to b0.  The engine only ever
    reads and writes its own context's buffers.
    """

    def __init__(self, ct, cbct_shifted, qmax, norm_planes, device=0, **kw):
        p = disc.make_params(global_shift=False, quant_max=tuple(qmax), norm_planes=tuple(norm_planes), **kw)
        self.reg = disc.Registration(p, device=device)
        self.reg.set_images(ct, cbct_shifted)
        self.device = ct.device
        self.shape = tuple(ct.shape)

    def close(self):
        self.reg.close()

    def level_shape(self, level):
        """(nz, ny, nx) of this slab's buffer at pyramid level `level`."""
        nz, ny, nx = self.shape
        for _ in range(level):
            nz, ny, nx = (nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2
        return nz, ny, nx

    def iterate_once(self, level):
        """One iteration at `level`; the interior sums (sum |dr|, sum |r|) of it."""
        self.reg.iterate(1, sync=False)
        s = self.reg.norm_sums(level, cap=1)     # set_level_field restarts the count
        return float(s[0, 0]), float(s[0, 1])

    def level_field(self, level):
        import torch
        nz, ny, nx = self.level_shape(level)
        f = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=self.device)
        return self.reg.get_level_field(level, f)

    def set_level_field(self, level, field):
        self.reg.set_field(level, field.contiguous())

    def upsample(self, level):
        """This slab's buffer field at `level` up-sampled to level - 1 (Algorithm A1)."""
        import torch
        nz, ny, nx = self.level_shape(level - 1)
        rf = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=self.device)
        disc.k_upsample_field2(self.level_field(level), rf)
        return rf


def run_slab_rank(engine, plan, rank, nz, levels, iters, dist, stop_eps=0.0, stop_window=10, group=None,
                  sums_device="cpu"):
    """Algorithm A1 for slab `rank` of `plan` (slab_plan over the finest level's
    nz planes), one slab per rank: per iteration the engine's step on the rank's
    buffer, the allreduce of the interior norm sums (allreduce_norm_sums), the
    stop rule of Sec. 2.3 on the summed history (disc_norm_stop_rule; every rank
    decides alike), and the halo exchange (halo_exchange); at a level's end each
    rank up-samples its own buffer and the finer level starts with an exchange.
    ``iters`` coarsest first.  Returns the summed norm sums per level (finest
    first), [k][2] float64 each.  `engine` provides iterate_once(level) ->
    (sum |dr|, sum |r|), level_field(level), set_level_field(level, field) and
    upsample(level) (LibdiscSlab on a GPU; the tests drive the FP64 oracle
    through the same calls on CPU ranks).  ``dist`` None: a single rank (one
    slab, no collectives)."""
    import torch
    hist = [[] for _ in range(levels)]
    for level in range(levels - 1, -1, -1):
        lplan = level_plan(plan, nz, level)
        for _ in range(iters[levels - 1 - level]):
            sdr, sr = engine.iterate_once(level)
            if dist is not None:
                sums = torch.tensor([sdr, sr], dtype=torch.float64, device=sums_device)
                allreduce_norm_sums(sums, dist, group)
                sdr, sr = float(sums[0]), float(sums[1])
            hist[level].append((sdr, sr))
            _, stop = disc.norm_stop_rule(hist[level], stop_window, stop_eps)
            if dist is not None:
                buf = engine.level_field(level)
                halo_exchange(lplan, rank, buf, dist, group)
                engine.set_level_field(level, buf)
            if stop:
                break
        if level > 0:
            fine = engine.upsample(level)
            if dist is not None:
                halo_exchange(level_plan(plan, nz, level - 1), rank, fine, dist, group)
            engine.set_level_field(level - 1, fine)
    return [np.array(h, np.float64).reshape(-1, 2) for h in hist]

