#!/usr/bin/env python
"""DISC hot-path benchmark: voxel-iterations per second on one B300.

A step is one full DISC registration schedule (Algorithm A1) of a synthetic
CT/CBCT pair already resident in HBM: the field is reset at the coarsest level
and every iteration of every level runs (warp, patch moments, correction,
force, update, Gaussian, convergence norm; field up-sampling between levels).
The metric is the total number of voxel-iterations of the schedule divided by
the step time (CUDA events on the library's stream, after warm-up).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # the head-and-neck-sized pair: 256x256x128, patch 11^3, sigma 1.5, 3 levels x 100 iterations
    "headneck-256x256x128": dict(dims=(256, 256, 128), patch=(11, 11, 11), sigma=1.5, levels=3,
                                 iters=(100, 100, 100), gen="head_neck"),
    # the small ellipsoid pair: 64x64x32, patch 7^3, sigma 1, 1 level x 50 iterations
    "ellipsoid-64x64x32": dict(dims=(64, 64, 32), patch=(7, 7, 7), sigma=1.0, levels=1, iters=(50,),
                               gen="ellipsoid"),
    # the large pair: 512x512x256, patch 15^3, sigma 2, 4 levels x 200 iterations
    "large-512x512x256": dict(dims=(512, 512, 256), patch=(15, 15, 15), sigma=2.0, levels=4,
                              iters=(200, 200, 200, 200), gen="head_neck"),
}
DEFAULT_WORKLOAD = "large-512x512x256"
CONTINUITY_WORKLOAD = "headneck-256x256x128"   # timed beside the headline as a second plain form
METRIC = "Gvoxel-iterations/s and % of HBM roofline, plain vs batched/adjoint form, 1 B300"
UNIT = "Gvoxel-it/s"
BOX_BYTES_PER_VOXEL = 32     # moments/force pass: read m (4) + zs (4) + r (12), write u (12)
GAUSS_BYTES_PER_VOXEL = 24   # Gaussian (field in and out, 12 + 12)
WARP_BYTES_PER_VOXEL = 20    # warp: read r (12) + I_m (4, taps amortised), write m (4)


def level_dims(dims, levels):
    out = [tuple(dims)]
    for _ in range(1, levels):
        out.append(tuple((d + 1) // 2 for d in out[-1]))
    return out


def schedule_units(w):
    """Voxel-iterations of one full schedule (coarsest level first in iters)."""
    dims = level_dims(w["dims"], w["levels"])
    tot = 0
    for lev in range(w["levels"]):
        nx, ny, nz = dims[lev]
        tot += nx * ny * nz * w["iters"][w["levels"] - 1 - lev]
    return tot


def make_pair(w):
    from paper_1204_6295_b300 import phantom
    nx, ny, nz = w["dims"]
    if w["gen"] == "ellipsoid":
        return phantom.ellipsoid_pair(nx, ny, nz)
    return phantom.head_neck_pair(nx, ny, nz)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


ROOFLINE_SOURCES = ("box_wide.cu", "box_tma.cu", "box_dev.cuh", "box_pass.cu", "tma_dev.cuh")   # the pass and its planner


def source_digest():
    """Digest of the sources that define the roofline kernel (its counters go stale with them)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1204_6295_b300", "csrc")
    for name in ROOFLINE_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    with open(os.path.join(ROOT, "paper_1204_6295_b300", "build.py"), "rb") as f:   # the compile flags
        h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload):
    """DRAM bytes per launch of the pass-A kernel from a committed ncu summary, if current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[workload]
        if e.get("source_digest") != source_digest():
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cpu():
    """The host the oracle is timed on: logical CPUs and the CPU model."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or None
    return {"nproc": os.cpu_count(), "cpu": model}


def host_cores():
    """Logical CPUs this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


ORACLE_BLOCK = (128, 128, 32)   # (x, y, z) interior of one worker's block of the finest level


def _oracle_block_job(job):
    """Worker process: `iters` oracle iterations (from r = 0) on one block of the
    finest level, its z interior plus a halo of planes on each side (the halo is
    the reach of one iteration: Gaussian radius, patch half size, one plane of
    the gradient); returns (interior voxel-iterations, seconds)."""
    ct, Is, patch, sigma, iters, interior = job
    import numpy as np
    from oracle import disc_oracle as O
    P = O.Params(patch=patch, sigma=sigma, levels=1, iters=[1])
    r = np.zeros((3,) + ct.shape)
    t0 = time.perf_counter()
    for _ in range(iters):
        r, _, _, _ = O.iteration(ct, Is, r, P)
    return interior * iters, time.perf_counter() - t0


def _noop(_):
    return 0


def oracle_blocks(w, pair, n_jobs):
    """Jobs for the multi-core oracle timing: blocks of ORACLE_BLOCK voxels (x, y
    crops of the finest level, z slabs with the one-iteration halo) taken in
    order over the volume."""
    import math

    import numpy as np
    from oracle import disc_oracle as O
    nx, ny, nz = w["dims"]
    bx, by, bz = (min(b, n) for b, n in zip(ORACLE_BLOCK, (nx, ny, nz)))
    R = int(math.ceil(3.0 * w["sigma"]))
    halo = R + (w["patch"][2] - 1) // 2 + 1
    Is, _ = O.global_shift(pair.ct, pair.cbct)
    jobs = []
    for z0 in range(0, nz - bz + 1, bz):
        for y0 in range(0, ny - by + 1, by):
            for x0 in range(0, nx - bx + 1, bx):
                if len(jobs) == n_jobs:
                    return jobs, halo
                za, zb = max(0, z0 - halo), min(nz, z0 + bz + halo)
                sl = (slice(za, zb), slice(y0, y0 + by), slice(x0, x0 + bx))
                jobs.append((np.ascontiguousarray(pair.ct[sl], np.float64),
                             np.ascontiguousarray(Is[sl]), tuple(w["patch"]), w["sigma"], 1, bx * by * bz))
    return jobs, halo


def oracle_all_cores(w, pair, iters=4, pool=None):
    """The FP64 oracle timed on every host core: one spawned process per core,
    each running `iters` iterations on its own block of the finest level.
    Returns (Gvoxel-it/s over the interiors, cores, sample text, seconds)."""
    import multiprocessing as mp
    cores = host_cores()
    jobs, halo = oracle_blocks(w, pair, cores)
    jobs = [j[:4] + (iters,) + j[5:] for j in jobs]
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(len(jobs))
        pool.map(_noop, range(len(jobs)))      # process start and imports outside the timing
    try:
        t0 = time.perf_counter()
        res = pool.map(_oracle_block_job, jobs, chunksize=1)
        el = time.perf_counter() - t0
    finally:
        if own:
            pool.close()
            pool.join()
    units = sum(r[0] for r in res)
    bx, by, bz = (min(b, n) for b, n in zip(ORACLE_BLOCK, w["dims"]))
    sample = (f"{len(jobs)} processes (one per logical CPU), each {iters} oracle iteration(s) from r = 0 on "
              f"its own {bx}x{by}x{bz} block of the finest level plus {halo} halo planes per side in z "
              f"(halo work not counted), numpy float64, {el:.1f} s wall")
    return units / el / 1e9, len(jobs), sample, el


def cpu_baseline(w, pair, budget_s=8.0):
    """The FP64 oracle timed on this host: every core (one process per core,
    blocks of the finest level), and one thread on a z-slab of the finest level."""
    import numpy as np
    from oracle import disc_oracle as O
    nx, ny, nz = w["dims"]
    planes = max(1, min(nz, (2 << 20) // (nx * ny)))
    P = O.Params(patch=w["patch"], sigma=w["sigma"], levels=1, iters=[1])
    Is, _ = O.global_shift(pair.ct, pair.cbct)
    ct = pair.ct[:planes].astype(np.float64)
    Is = Is[:planes]
    r = np.zeros((3,) + ct.shape)
    n_vox = ct.size
    t0 = time.perf_counter()
    its = 0
    while True:
        r, _, _, _ = O.iteration(ct, Is, r, P)
        its += 1
        el = time.perf_counter() - t0
        if el >= budget_s or its >= 50:
            break
    single = its * n_vox / el / 1e9
    value, cores, sample, _ = oracle_all_cores(w, pair)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_cpu(),
            "sample": sample,
            "single_thread": {"value": single, "unit": UNIT, "cores": 1,
                              "sample": f"{its} oracle iterations on the first {planes} z-planes "
                                        f"({nx}x{ny}x{planes}) of the finest level, numpy float64, one "
                                        f"thread, {el:.1f} s"}}


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    import multiprocessing as mp
    pair = make_pair(w)
    cores = host_cores()
    jobs, halo = oracle_blocks(w, pair, cores)
    pool = mp.get_context("spawn").Pool(len(jobs))
    pool.map(_noop, range(len(jobs)))
    try:
        for _ in range(args.warmup):
            pool.map(_oracle_block_job, jobs, chunksize=1)
        t0 = time.perf_counter()
        units = 0
        for _ in range(args.steps):
            units += sum(r[0] for r in pool.map(_oracle_block_job, jobs, chunksize=1))
        el = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    value = units / el / 1e9
    bx, by, bz = (min(b, n) for b, n in zip(ORACLE_BLOCK, w["dims"]))
    sample = (f"each step = one oracle iteration (warp, moments, correction, force, Gaussian) from r = 0 in "
              f"each of {len(jobs)} processes (one per logical CPU), each on its own {bx}x{by}x{bz} block of "
              f"the finest level plus {halo} halo planes per side in z (halo work not counted), numpy float64")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "dims": list(w["dims"]), "patch": list(w["patch"]),
                       "sigma": w["sigma"], "levels": w["levels"], "iters": list(w["iters"]),
                       "sample_block": [bx, by, bz], "sample_halo_planes": halo},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": len(jobs), "kind": "oracle",
                             "host": host_cpu(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_kernels(disc, torch, w, pair_dev, field_dev, reps=20):
    """CUDA-event timing of the per-iteration kernels at the finest level.

    Each is launched through its kernel-level entry point on the current torch
    stream, with the launch configuration the schedule uses (the plan depends
    only on sizes and patch).  Returns seconds per launch.
    """
    nx, ny, nz = w["dims"]
    N = nx * ny * nz
    ct, cbct = pair_dev
    patch = w["patch"]
    qs_s = disc.qscale(float(cbct.abs().max()), patch)
    qs_m = disc.qscale(float(ct.abs().max()), patch)
    zs, m = torch.empty_like(ct), torch.empty_like(ct)
    disc.k_static_norm(cbct, zs, patch, qs_s)
    disc.k_warp(ct, field_dev, m)
    u = torch.empty_like(field_dev)
    r2 = torch.empty_like(field_dev)
    s = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps / 1e3

    return {"box_s": timed(lambda: disc.k_force_update(m, zs, field_dev, u, patch, qs_m)),
            "gauss_s": timed(lambda: disc.k_gauss(u, r2, w["sigma"])),
            "warp_s": timed(lambda: disc.k_warp(ct, field_dev, m)),
            "N": N, "zs": zs, "qs_m": qs_m}


def time_differentiable(disc, torch, w, pair_dev, field_dev, kt, reps=5):
    """Forward (loss) + backward (adjoint gradient) of the SSD form at the finest level."""
    ct, _ = pair_dev
    patch = w["patch"]
    if len(set(patch)) != 1:
        return None
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(field_dev)
    s = torch.cuda.current_stream()

    def step():                               # loss and gradient from one adjoint pass
        disc.k_ssd_grad(ct, kt["zs"], field_dev, grad, patch, kt["qs_m"], loss_out=loss)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / reps / 1e3
    return {"value": kt["N"] / t / 1e9, "unit": "Gvoxel-evaluations/s (forward + backward)",
            "ms_per_step": t * 1e3, "algorithmic_bytes_per_voxel": 32,
            "what": "disc_k_ssd_grad with loss_out on the finest level (256x256x128 for the default "
                    "workload): warp, moments, loss and adjoint coefficients in one pass, their box sums, "
                    "the warp's adjoint; patch statistics recomputed, not stored"}


def time_masked(disc, torch, w, pair_dev, dist, steps=1):
    """The same schedule with the mask and fill of Eqs. 7-10 on (mask_mode 1)."""
    ct, cbct = pair_dev
    nx, ny, nz = w["dims"]
    reg = disc.Registration(patch=w["patch"], sigma=w["sigma"], levels=w["levels"], iters=w["iters"],
                            mask_mode=1)
    reg.set_images(ct, cbct)
    hu0, a_m = reg.mask_constants()
    cx, cy, cz = level_dims(w["dims"], w["levels"])[-1]
    zeros = torch.zeros((3, cz, cy, cx), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()

    def step():
        reg.set_field(w["levels"] - 1, zeros)
        reg.iterate(-1, sync=False)

    step()                                        # warm-up (captures the graphs)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    t = reduce_max(dist, e0.elapsed_time(e1) / steps / 1e3)
    reg.close()
    world = dist.get_world_size() if dist else 1
    return {"value": job_throughput(schedule_units(w), world, t), "unit": UNIT, "ms_per_step": t * 1e3,
            "hu0": hu0, "a_m": a_m,
            "what": "the plain workload with the xi mask of Eq. 7 and the Jacobi fill of Eqs. 8-10 "
                    "every iteration (HU0 = 2|dHU|, a in [0.5, 1.5] a_m, T 7x7x3, h 50 HU, <= 32 passes)"}


BATCH_PAIRS_PER_RANK = 16
BATCH_WORKLOAD = dict(patch=(9, 9, 9), sigma=1.5, levels=3, iters=(100, 100, 100))


def time_batched(disc, torch, dist, steps=2):
    """The batched workload: 16 pairs of uneven size advanced together, against
    the plain per-pair loop over the same pairs (separate contexts, one after the
    other), both timed with CUDA events on the current stream."""
    from paper_1204_6295_b300 import phantom, shard
    bw = BATCH_WORKLOAD
    world = dist.get_world_size() if dist else 1
    rank = dist.get_rank() if dist else 0
    # 16 pairs per rank (weak scaling), sharded across ranks by the
    # longest-processing-time rule on their voxel-iterations; no exchange
    n_pairs = BATCH_PAIRS_PER_RANK * world
    sizes = phantom.batch_sizes(n_pairs)
    loads = [schedule_units(dict(bw, dims=d)) for d in sizes]
    share = shard.lpt_assign(loads, world)
    images = phantom.batch_pair_images(n_pairs, indices=share[rank])
    units = sum(loads)                            # the whole job's voxel-iterations
    s = torch.cuda.current_stream()

    def timed(step):
        step()                                    # warm-up (the batch also tunes here)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            step()
        e1.record(s)
        torch.cuda.synchronize()
        return reduce_max(dist, e0.elapsed_time(e1) / steps / 1e3)

    batch = disc.Batch(len(images), **bw)
    for i, (ct, cbct) in enumerate(images):
        batch.set_images(i, ct, cbct)

    def batch_step():
        batch.restart()
        batch.iterate(-1)

    t_batch = timed(batch_step)
    tuning = [batch.tuning(l) for l in range(bw["levels"])]
    gauss_tuning = [batch.gauss_tuning(l) for l in range(bw["levels"])]
    box_paths = [batch.box_path(l) for l in range(bw["levels"])]
    batch.close()
    regs = []
    for ct, cbct in images:
        reg = disc.Registration(**bw)
        reg.set_images(ct, cbct)
        nz, ny, nx = ct.shape
        cz, cy, cx = level_dims((nx, ny, nz), bw["levels"])[-1][::-1]
        regs.append((reg, torch.zeros((3, cz, cy, cx), dtype=torch.float32, device="cuda")))

    def loop_step():
        for reg, z in regs:
            reg.set_field(bw["levels"] - 1, z)
            reg.iterate(-1, sync=False)

    t_loop = timed(loop_step)
    for reg, _ in regs:
        reg.close()
    return {"value": units / t_batch / 1e9, "unit": UNIT,
            "plain_loop_value": units / t_loop / 1e9,
            "speedup_vs_plain_loop": t_loop / t_batch, "ms_per_step": t_batch * 1e3,
            "plain_loop_ms_per_step": t_loop * 1e3, "voxel_iterations_per_step": units,
            "pairs": [list(d) for d in sizes],
            "pairs_per_rank": [len(x) for x in share],
            "max_over_mean_rank_load": max(shard.rank_loads(loads, share)) * world / units,
            "tuning_items_grid_zmult_per_level_fine_first": tuning,
            "box_path_per_level_fine_first": box_paths,
            "gauss_zlen_separate_warp_per_level_fine_first": gauss_tuning,
            "what": "16 head-and-neck pairs (2s, 2s, s) per rank, s in 64..160, patch 9^3, "
                    "sigma 1.5, 3 levels x 100 iterations, pairs sharded across ranks by the "
                    "longest-processing-time rule (no exchange): disc_batch (one launch per step "
                    "over a rank's pairs, graph per level) vs its pairs' separate contexts run one "
                    "after the other; value = all ranks' voxel-iterations / slowest rank's time"}


def time_plain(disc, torch, w, dist, steps=5, warmup=2, pair_dev=None, switches=0):
    """A plain workload's full schedule: another workload (a second line of the
    plain form), or the same one with test switches (an alternative schedule)."""
    if pair_dev is None:
        pair = make_pair(w)
        ct = torch.from_numpy(pair.ct).cuda()
        cbct = torch.from_numpy(pair.cbct).cuda()
    else:
        ct, cbct = pair_dev
    cnx, cny, cnz = level_dims(w["dims"], w["levels"])[-1]
    zeros = torch.zeros((3, cnz, cny, cnx), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    with disc.test_switches(switches):
        reg = disc.Registration(patch=w["patch"], sigma=w["sigma"], levels=w["levels"], iters=w["iters"])
    with reg:
        reg.set_images(ct, cbct)

        def step():
            reg.set_field(w["levels"] - 1, zeros)
            reg.iterate(-1, sync=False)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            step()
        e1.record(s)
        torch.cuda.synchronize()
    t = reduce_max(dist, e0.elapsed_time(e1) / steps / 1e3)
    world = dist.get_world_size() if dist else 1
    return {"value": job_throughput(schedule_units(w), world, t), "unit": UNIT, "ms_per_step": t * 1e3,
            "steps": steps, "dims": list(w["dims"]), "patch": list(w["patch"]), "sigma": w["sigma"],
            "levels": w["levels"], "iters_coarse_to_fine": list(w["iters"]),
            "voxel_iterations_per_step": schedule_units(w)}


MIXED_HEADNECK_PAIRS = 4


def time_mixed_batch(disc, torch, w, pair_dev, dist, steps=1):
    """The large pair batched with four head-and-neck-sized pairs (256x256x128)
    under the large pair's parameters, against the same five pairs run one
    after the other as separate contexts."""
    from paper_1204_6295_b300 import phantom
    hn = [(256, 256, 128)] * MIXED_HEADNECK_PAIRS
    images = [pair_dev] + [(torch.from_numpy(c).cuda(), torch.from_numpy(b).cuda())
                           for c, b in phantom.batch_pair_images(len(hn), sizes=hn)]
    dims = [tuple(w["dims"])] + hn
    units = sum(schedule_units(dict(w, dims=d)) for d in dims)
    kw = dict(patch=w["patch"], sigma=w["sigma"], levels=w["levels"], iters=w["iters"])
    s = torch.cuda.current_stream()

    def timed(step):
        step()                                    # warm-up (graphs, tuning)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            step()
        e1.record(s)
        torch.cuda.synchronize()
        return reduce_max(dist, e0.elapsed_time(e1) / steps / 1e3)

    batch = disc.Batch(len(images), **kw)
    for i, (ct, cbct) in enumerate(images):
        batch.set_images(i, ct, cbct)

    def batch_step():
        batch.restart()
        batch.iterate(-1)

    t_batch = timed(batch_step)
    batch.close()
    regs = []
    for ct, cbct in images:
        reg = disc.Registration(**kw)
        reg.set_images(ct, cbct)
        nz, ny, nx = ct.shape
        cz, cy, cx = level_dims((nx, ny, nz), w["levels"])[-1][::-1]
        regs.append((reg, torch.zeros((3, cz, cy, cx), dtype=torch.float32, device="cuda")))

    def loop_step():
        for reg, z in regs:
            reg.set_field(w["levels"] - 1, z)
            reg.iterate(-1, sync=False)

    t_loop = timed(loop_step)
    for reg, _ in regs:
        reg.close()
    world = dist.get_world_size() if dist else 1
    return {"value": job_throughput(units, world, t_batch), "unit": UNIT,
            "plain_loop_value": job_throughput(units, world, t_loop),
            "speedup_vs_plain_loop": t_loop / t_batch, "ms_per_step": t_batch * 1e3,
            "plain_loop_ms_per_step": t_loop * 1e3, "voxel_iterations_per_step": units,
            "pairs": [list(d) for d in dims],
            "what": "the large pair and four 256x256x128 head-and-neck pairs in one disc_batch "
                    "(patch, sigma and schedule of the large pair) vs the five pairs' separate "
                    "contexts one after the other; every rank runs the same five pairs"}


def reduce_max(dist, seconds, device="cuda"):
    """Largest value over the ranks of the process group (the step time of the job)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job Gvoxel-iterations/s: every rank processes units_per_rank per step (weak scaling)."""
    return world * units_per_rank / seconds / 1e9


def run_ours(args, w, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1204_6295_b300 import disc
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    pair = make_pair(w)
    nx, ny, nz = w["dims"]
    dims = level_dims(w["dims"], w["levels"])
    cnx, cny, cnz = dims[-1]
    ct = torch.from_numpy(pair.ct).cuda()
    cbct = torch.from_numpy(pair.cbct).cuda()
    zeros_coarse = torch.zeros((3, cnz, cny, cnx), dtype=torch.float32, device="cuda")
    reg = disc.Registration(patch=w["patch"], sigma=w["sigma"], levels=w["levels"], iters=w["iters"])
    reg.set_images(ct, cbct)
    units = schedule_units(w)
    L = w["levels"]

    def step():
        reg.set_field(L - 1, zeros_coarse)
        reg.iterate(-1, sync=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = reg.launch_count()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = reg.launch_count() - launches0     # kernels disc_iterate launched in the timed steps
    ms = reduce_max(dist, e0.elapsed_time(e1) / args.steps)
    value = job_throughput(units, world, ms / 1e3)

    # kernel timing for the roofline at the finest level, on the final field
    field = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    reg.get_field(field)
    kt = time_kernels(disc, torch, w, (ct, cbct), field)
    diff_form = time_differentiable(disc, torch, w, (ct, cbct), field, kt)
    peak, peak_kind = load_peaks()
    box_gbs = BOX_BYTES_PER_VOXEL * kt["N"] / kt["box_s"] / 1e9
    gauss_gbs = GAUSS_BYTES_PER_VOXEL * kt["N"] / kt["gauss_s"] / 1e9
    warp_gbs = WARP_BYTES_PER_VOXEL * kt["N"] / kt["warp_s"] / 1e9
    traffic = recorded_traffic(args.workload)

    continuity = (time_plain(disc, torch, WORKLOADS[CONTINUITY_WORKLOAD], dist)
                  if args.workload != CONTINUITY_WORKLOAD else None)
    # the same schedule with the next iteration's warp in a kernel of its own
    # at every level (the default runs it inside the Gaussian's xy pass)
    sep = time_plain(disc, torch, w, dist, steps=min(args.steps, 3), warmup=1, pair_dev=(ct, cbct),
                     switches=disc.SW_SEPARATE_WARP)
    warp_placement = {"default_fused_in_gauss_xy_ms": ms,
                      "separate_kernel_everywhere_ms": sep["ms_per_step"],
                      "what": "whole schedule: the warp of I_m by the new field inside the Gaussian's last "
                              "pass (the xy pass, r in registers), or as a kernel of its own after the "
                              "Gaussian (a thread marches a column in z and loads the field two planes ahead "
                              "of its gathers)"}
    batched = None if args.no_batched else time_batched(disc, torch, dist)
    masked = time_masked(disc, torch, w, (ct, cbct), dist)
    mixed = (time_mixed_batch(disc, torch, w, (ct, cbct), dist)
             if args.workload == "large-512x512x256" and not args.no_batched else None)

    # end to end through the public API with host buffers (pinned)
    ct_h = torch.from_numpy(pair.ct).pin_memory()
    cbct_h = torch.from_numpy(pair.cbct).pin_memory()
    out_h = torch.empty((3, nz, ny, nx), dtype=torch.float32).pin_memory()
    ct_np, cbct_np, out_np = ct_h.numpy(), cbct_h.numpy(), out_h.numpy()
    e2e_steps = max(1, min(args.steps, 3))
    reg.set_images(ct_np, cbct_np)
    reg.iterate(-1, sync=False)
    reg.get_field(out_np)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        reg.set_images(ct_np, cbct_np)
        reg.iterate(-1, sync=False)
        reg.get_field(out_np)
    torch.cuda.synchronize()
    e2e_s = reduce_max(dist, (time.perf_counter() - t0) / e2e_steps)
    e2e = {"value": job_throughput(units, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(2 * nx * ny * nz * 4), "d2h_bytes_per_step": int(3 * nx * ny * nz * 4),
           "ms_per_step": e2e_s * 1e3,
           "what": "disc_set_images(host CT, CBCT) + disc_iterate(full schedule) + disc_get_field(host)"}
    reg.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "dims": list(w["dims"]), "patch": list(w["patch"]),
                   "sigma": w["sigma"], "levels": w["levels"], "iters_coarse_to_fine": list(w["iters"]),
                   "voxel_iterations_per_step": units, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2: finest-level working set "
                         f"{(9 * nx * ny * nz * 4) / 1e6:.0f} MB > 126 MB"},
        "roofline": {"bound": "hbm",
                     "kernel": "the iteration pass at the finest level (patch moments, correction, force, update): "
                               "k_box_wide (32 x 32 tiles, balanced z shares, bulk-tensor-copy fed) where the "
                               "planner picks it, as on the 512x512x256 and 256x256x128 finest levels",
                     "achieved": box_gbs, "peak": peak, "unit": "GB/s", "frac": box_gbs / peak,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "traffic": traffic, "algorithmic_bytes_per_voxel": BOX_BYTES_PER_VOXEL,
                     "launch_ms": kt["box_s"] * 1e3,
                     "note": "issue-bound (exact 64-bit patch sums), not HBM-bound; see profiles/"},
        "kernels": {"gauss_xy_plus_z": {"achieved_gbs": gauss_gbs, "frac": gauss_gbs / peak,
                                        "launch_ms": kt["gauss_s"] * 1e3,
                                        "algorithmic_bytes_per_voxel": GAUSS_BYTES_PER_VOXEL},
                    "warp": {"achieved_gbs": warp_gbs, "frac": warp_gbs / peak, "launch_ms": kt["warp_s"] * 1e3,
                             "algorithmic_bytes_per_voxel": WARP_BYTES_PER_VOXEL}},
        "forms": {"plain": {"value": value, "unit": UNIT},
                  **({"plain_" + CONTINUITY_WORKLOAD: continuity} if continuity else {}),
                  "warp_placement": warp_placement,
                  "batched": batched,
                  "differentiable": diff_form,
                  "masked": masked,
                  **({"batched_with_headneck": mixed} if mixed else {}),
                  "effective_hbm_frac_32B_model": value * 1e9 * 32 / (peak * 1e9)},
        "e2e": e2e,
        "gpu_launches": launches,
        "gpu_launches_source": "disc_get_launch_count over the timed steps: kernel nodes of each "
                               "replayed level graph plus the up-sampling launches",
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, pair)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_slab_split(args, w, rank, world, local_rank):
    """One volume split into z slabs, one slab per rank (slab.run_slab_rank):
    per iteration each rank's context advances its slab, the interior norm sums
    are added over the ranks (NCCL allreduce) and the halo planes of the field
    are exchanged point to point into each rank's own buffer.  Strong scaling:
    value = the whole volume's voxel-iterations / the slowest rank's time."""
    import torch
    from paper_1204_6295_b300 import disc, slab
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pair = make_pair(w)                           # every rank draws the same seeded volume
    nx, ny, nz = w["dims"]
    L = w["levels"]
    ct = torch.from_numpy(pair.ct).cuda()
    cbct = torch.from_numpy(pair.cbct).cuda()
    shifted = torch.empty_like(cbct)
    disc.k_global_shift(ct, cbct, shifted)        # Sec. 2.3: over the whole volume
    mx = torch.empty(2, dtype=torch.float32, device="cuda")
    disc.k_max_abs(ct, mx[0:1])
    disc.k_max_abs(shifted, mx[1:2])
    qmax = [float(v) for v in mx.cpu()]
    halo = slab.halo_planes(w["patch"], w["sigma"], 0, 8.0, L)
    plan = slab.slab_plan(nz, world, halo, 1 << (L - 1))
    z0, z1, b0, b1 = plan[rank]
    eng = slab.LibdiscSlab(ct[b0:b1].contiguous(), shifted[b0:b1].contiguous(), qmax, (z0 - b0, z1 - b0),
                           device=local_rank, patch=w["patch"], sigma=w["sigma"], levels=L, iters=w["iters"])
    del ct, cbct, shifted
    cz, cy, cx = eng.level_shape(L - 1)
    zeros = torch.zeros((3, cz, cy, cx), dtype=torch.float32, device="cuda")

    def step():
        eng.set_level_field(L - 1, zeros)
        slab.run_slab_rank(eng, plan, rank, nz, L, w["iters"], dist, sums_device="cuda")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    ms = reduce_max(dist, e0.elapsed_time(e1) / args.steps)
    eng.close()
    if rank == 0:
        units = schedule_units(w)
        print(json.dumps({
            "metric": METRIC, "value": units / (ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "dims": list(w["dims"]), "patch": list(w["patch"]),
                       "sigma": w["sigma"], "levels": L, "iters_coarse_to_fine": list(w["iters"]),
                       "voxel_iterations_per_step": units, "parallelism": f"z-slabs x{world}",
                       "halo_planes": halo, "split": "slab"},
            "what": "one volume in z slabs, one per rank: per iteration a context step on each slab, an "
                    "allreduce of the interior norm sums and a point-to-point halo exchange"}), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_once(w):
    """One launch of each per-iteration kernel at the finest level (for ncu captures).

    Launch order: static patch normalisation, warp, box pass (iteration mode),
    Gaussian z pass, Gaussian xy pass; then a one-level context's set-up and
    two iterations (warp, then per iteration the box pass, the Gaussian z
    pass, the Gaussian xy pass with the fused warp and the norm).
    """
    import torch
    from paper_1204_6295_b300 import disc
    pair = make_pair(w)
    nx, ny, nz = w["dims"]
    ct = torch.from_numpy(pair.ct).cuda()
    cbct = torch.from_numpy(pair.cbct).cuda()
    r = torch.from_numpy(pair.u_true).cuda()        # a realistic smooth field
    patch = w["patch"]
    qs_s = disc.qscale(float(cbct.abs().max()), patch)
    qs_m = disc.qscale(float(ct.abs().max()), patch)
    zs, m = torch.empty_like(ct), torch.empty_like(ct)
    u, r2 = torch.empty_like(r), torch.empty_like(r)
    disc.k_static_norm(cbct, zs, patch, qs_s)
    disc.k_pass_a(ct, zs, r, u, patch, qs_m, m_out=m)
    disc.k_gauss(u, r2, w["sigma"])
    # then two iterations of the finest level as the schedule runs them (box pass,
    # Gaussian xy, Gaussian z with the fused warp, norm), in a one-level context
    with disc.Registration(patch=patch, sigma=w["sigma"], levels=1, iters=(2,)) as reg:
        reg.set_images(ct, cbct)
        reg.iterate(-1, sync=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_once": True, "workload": [nx, ny, nz], "patch": list(patch)}))
    return 0


def run_profile_schedule(w):
    """One whole schedule of the workload from a zero field (for launch lists):
    set-up, then every level's iterations as the timed steps run them."""
    import torch
    from paper_1204_6295_b300 import disc
    pair = make_pair(w)
    ct = torch.from_numpy(pair.ct).cuda()
    cbct = torch.from_numpy(pair.cbct).cuda()
    with disc.Registration(patch=w["patch"], sigma=w["sigma"], levels=w["levels"], iters=w["iters"]) as reg:
        reg.set_images(ct, cbct)
        reg.iterate(-1, sync=False)
        torch.cuda.synchronize()
        launches = reg.launch_count()
    print(json.dumps({"profile_schedule": True, "workload": list(w["dims"]), "launches": launches}))
    return 0


def run_profile_batched():
    """The batched workload's 16 pairs (for launch lists): one schedule that also
    tunes each level, then a second one, as the timed steps run it, inside the
    NVTX range "profiled batch schedule" (ncu --nvtx --nvtx-include selects it)."""
    import torch
    from paper_1204_6295_b300 import disc, phantom
    bw = BATCH_WORKLOAD
    sizes = phantom.batch_sizes(BATCH_PAIRS_PER_RANK)
    images = phantom.batch_pair_images(BATCH_PAIRS_PER_RANK)
    units = sum(schedule_units(dict(bw, dims=d)) for d in sizes)
    with disc.Batch(len(images), **bw) as batch:
        for i, (ct, cbct) in enumerate(images):
            batch.set_images(i, ct, cbct)
        batch.iterate(-1)                         # tunes every level
        batch.restart()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled batch schedule")
        batch.iterate(-1)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_batched": True, "pairs": [list(d) for d in sizes], "voxel_iterations": units}))
    return 0


def run_profile_masked(w, iters=2):
    """`iters` masked iterations (Eqs. 7-10) at the finest level only, from r = 0
    (for ncu captures of the fill passes): one context with one level."""
    import torch
    from paper_1204_6295_b300 import disc
    pair = make_pair(w)
    ct = torch.from_numpy(pair.ct).cuda()
    cbct = torch.from_numpy(pair.cbct).cuda()
    with disc.Registration(patch=w["patch"], sigma=w["sigma"], levels=1, iters=(iters,), mask_mode=1) as reg:
        reg.set_images(ct, cbct)
        done, _ = reg.iterate(-1)
    torch.cuda.synchronize()
    print(json.dumps({"profile_masked": True, "workload": list(w["dims"]), "iterations": done}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 16-pair batched form")
    ap.add_argument("--split", default="replicas", choices=["replicas", "slab"],
                    help="replicas: each rank runs the whole workload (weak scaling); slab: one volume "
                         "split into z slabs over the ranks (strong scaling)")
    ap.add_argument("--profile-once", action="store_true",
                    help="launch each per-iteration kernel once at the finest level and exit")
    ap.add_argument("--profile-schedule", action="store_true",
                    help="run one whole schedule of the workload and exit")
    ap.add_argument("--profile-masked", type=int, default=0, metavar="K",
                    help="run K masked iterations at the finest level and exit")
    ap.add_argument("--profile-batched", action="store_true",
                    help="run the 16-pair batched workload's schedule twice (the second in an NVTX range) "
                         "and exit")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus > 0 else 1)))
    if "WORLD_SIZE" not in os.environ:
        world = 1
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    w = WORKLOADS[args.workload]
    if args.profile_once:
        return run_profile_once(w)
    if args.profile_schedule:
        return run_profile_schedule(w)
    if args.profile_masked > 0:
        return run_profile_masked(w, args.profile_masked)
    if args.profile_batched:
        return run_profile_batched()
    if args.impl == "reference":
        return run_reference(args, w, rank, world)
    if args.split == "slab":
        return run_slab_split(args, w, rank, world, local_rank)
    return run_ours(args, w, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
