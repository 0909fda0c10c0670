"""Build libdisc.so (sm_103a) in-tree with nvcc.

``python -m paper_1204_6295_b300.build`` compiles every ``csrc/*.cu`` into
``paper_1204_6295_b300/libdisc.so``.  Objects are rebuilt only when a source
or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libdisc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


LIB_BOUNDS = os.path.join(HERE, "libdisc_bc.so")   # the bounds-checked build (-DDISC_BOUNDS_CHECK)


def build(verbose=False, force=False, extra_flags=(), bounds_check=False):
    """Compile libdisc.so, or with bounds_check=True the bounds-checked library
    libdisc_bc.so (every global index of the per-iteration kernels tested before
    its access; see disc_bounds_violations in include/disc.h)."""
    srcs = sources()
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    lib = LIB_BOUNDS if bounds_check else LIB
    if bounds_check:
        extra_flags = tuple(extra_flags) + ("-DDISC_BOUNDS_CHECK",)
    if not force and not _stale(lib, deps):
        return lib
    objdir = os.path.join(HERE, "_build_bc" if bounds_check else "_build")
    os.makedirs(objdir, exist_ok=True)
    objs, cmds = [], []
    # The normal build compiles each unit whole (-c): no device symbol crosses
    # units, and whole-unit code takes far fewer registers than relocatable
    # code (the xy Gaussian 40 against 80-96, the z-marching warp 40 against
    # 64).  The checked build shares one device counter between the units, so
    # it is relocatable (-dc) and device-linked.
    mode = "-dc" if bounds_check else "-c"
    for src in srcs:
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmds.append([_nvcc(), *ARCH, *NVCC_FLAGS, *extra_flags, "-I", INCLUDE, "-I", CSRC, mode, src, "-o", obj])
        objs.append(obj)
    if verbose:
        for cmd in cmds:
            print(" ".join(cmd), flush=True)
    # translation units compile independently: one nvcc per core
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        for done in ex.map(lambda c: subprocess.run(c, check=True), cmds):
            pass
    tmp = lib + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
    build(verbose=True, force="--force" in sys.argv, bounds_check=True)
