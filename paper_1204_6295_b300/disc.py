"""Python binding of libdisc.so (the C ABI in include/disc.h).

Argument marshalling only: every step of the registration runs in the CUDA
library.  Device buffers are torch CUDA tensors (float32, contiguous); host
buffers are numpy arrays.  Importing this module loads the library and fails
loudly if it has not been built (``python -m paper_1204_6295_b300.build``).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DISC_LIBRARY=bounds loads the bounds-checked build libdisc_bc.so instead
LIB_PATH = os.path.join(_HERE, "libdisc_bc.so" if os.environ.get("DISC_LIBRARY") == "bounds" else "libdisc.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "disc.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libdisc.so not found at {LIB_PATH}; build it with "
                      "`python -m paper_1204_6295_b300.build` (nvcc, sm_103a)")
_lib = ctypes.CDLL(LIB_PATH)

MEM_HOST, MEM_DEVICE = 0, 1
FORCE_THIRION, FORCE_DOUBLE = 0, 1
MAX_LEVELS = 8

STATUS = {0: "DISC_OK", 1: "DISC_ERR_ARG", 2: "DISC_ERR_SHAPE", 3: "DISC_ERR_STATE",
          4: "DISC_ERR_OOM", 5: "DISC_ERR_CUDA", 6: "DISC_ERR_TIMEOUT"}


class DiscError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.disc_status_str(status).decode()
        super().__init__(f"{where}: {msg}")


class Params(ctypes.Structure):
    _fields_ = [
        ("patch", ctypes.c_int32 * 3),
        ("gauss_sigma", ctypes.c_float),
        ("gauss_radius", ctypes.c_int32),
        ("levels", ctypes.c_int32),
        ("iters", ctypes.c_int32 * MAX_LEVELS),
        ("stop_eps", ctypes.c_float),
        ("stop_window", ctypes.c_int32),
        ("force_mode", ctypes.c_int32),
        ("global_shift", ctypes.c_int32),
        ("var_floor", ctypes.c_float),
        ("mask_mode", ctypes.c_int32),
        ("hu0_factor", ctypes.c_float),
        ("a_lo", ctypes.c_float),
        ("a_hi", ctypes.c_float),
        ("fill_h", ctypes.c_float),
        ("fill_t", ctypes.c_int32 * 3),
        ("fill_passes", ctypes.c_int32),
        ("smooth_mode", ctypes.c_int32),
        ("quant_max", ctypes.c_float * 2),
        ("norm_planes", ctypes.c_int32 * 2),
    ]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f32 = ctypes.c_float
_st = ctypes.c_int

_SIGS = {
    "disc_params_default": (_st, [ctypes.POINTER(Params)]),
    "disc_status_str": (ctypes.c_char_p, [_st]),
    "disc_create": (_st, [ctypes.POINTER(Params), ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "disc_set_images": (_st, [_vp, _vp, _vp, _i32, _i32, _i32, ctypes.c_int]),
    "disc_iterate": (_st, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_f32)]),
    "disc_get_field": (_st, [_vp, _vp, ctypes.c_int]),
    "disc_get_corrected": (_st, [_vp, _vp, ctypes.c_int]),
    "disc_set_field": (_st, [_vp, _i32, _vp, ctypes.c_int]),
    "disc_get_level_field": (_st, [_vp, _i32, _vp, ctypes.c_int]),
    "disc_get_progress": (_st, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "disc_get_norm_history": (_st, [_vp, _i32, _vp, _i32, ctypes.POINTER(_i32)]),
    "disc_get_norm_sums": (_st, [_vp, _i32, _vp, _i32, ctypes.POINTER(_i32)]),
    "disc_get_launch_count": (_st, [_vp, ctypes.POINTER(_i64)]),
    "disc_ssd": (_st, [_vp, _i32, _vp, ctypes.POINTER(ctypes.c_double), _vp, ctypes.c_int]),
    "disc_get_correction_means": (_st, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(_i64)]),
    "disc_norm_stop_rule": (_st, [_vp, _i32, _i32, _f32, _vp, ctypes.POINTER(_i32)]),
    "disc_destroy": (_st, [_vp]),
    "disc_qscale": (_f32, [_f32, ctypes.POINTER(_i32)]),
    "disc_batch_create": (_st, [ctypes.POINTER(Params), ctypes.c_int, _vp, _i32, ctypes.POINTER(_vp)]),
    "disc_batch_set_images": (_st, [_vp, _i32, _vp, _vp, _i32, _i32, _i32, ctypes.c_int]),
    "disc_batch_restart": (_st, [_vp]),
    "disc_batch_iterate": (_st, [_vp, _i32, ctypes.POINTER(_i32)]),
    "disc_batch_get_field": (_st, [_vp, _i32, _vp, ctypes.c_int]),
    "disc_batch_get_tuning": (_st, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "disc_batch_destroy": (_st, [_vp]),
    "disc_batch_get_box_path": (_st, [_vp, _i32, ctypes.POINTER(_i32)]),
    "disc_batch_pin_tuning": (_st, [_vp, _i32, _i32, _i32]),
    "disc_batch_get_gauss_tuning": (_st, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "disc_k_max_abs": (_st, [_vp, _i64, _vp, _vp]),
    "disc_k_global_shift": (_st, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "disc_k_downsample2": (_st, [_vp, _vp, _i32, _i32, _i32, _vp]),
    "disc_k_upsample_field2": (_st, [_vp, _vp, _i32, _i32, _i32, _vp]),
    "disc_k_static_norm": (_st, [_vp, _vp, _i32, _i32, _i32, ctypes.POINTER(_i32), _f32, _f32, _vp]),
    "disc_k_warp": (_st, [_vp, _vp, _vp, _i32, _i32, _i32, _vp]),
    "disc_k_pass_a": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32,
                            ctypes.POINTER(_i32), _f32, _f32, _i32, _vp]),
    "disc_k_pass_a_static": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32,
                                   ctypes.POINTER(_i32), _f32, _f32, _i32, _vp]),
    "disc_k_gauss": (_st, [_vp, _vp, _i32, _i32, _i32, _f32, _i32, _vp]),
    "disc_k_check_error": (_st, [_vp]),
    "disc_set_test_switches": (_st, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "disc_bounds_violations": (_st, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32)]),
    "disc_get_mask_constants": (_st, [_vp, ctypes.POINTER(_f32), ctypes.POINTER(_f32)]),
    "disc_k_static_stats": (_st, [_vp, _vp, _vp, _i32, _i32, _i32, ctypes.POINTER(_i32), _f32, _f32, _vp]),
    "disc_k_ratio_median": (_st, [_vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32, ctypes.POINTER(_i32), _f32, _f32,
                                  _vp]),
    "disc_k_correct_masked": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32,
                                    ctypes.POINTER(_i32), _f32, _f32, _f32, _f32, _f32, _f32,
                                    ctypes.POINTER(_i32), _i32, _vp]),
    "disc_k_force": (_st, [_vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp]),
    "disc_k_nmi": (_st, [_vp, _vp, _i64, _i32, _vp, _vp]),
    "disc_k_canny": (_st, [_vp, _vp, _i32, _i32, _i32, _f32, _f32, _f32, _vp]),
    "disc_k_edge_rmse": (_st, [_vp, _vp, _i64, _vp, _vp]),
    "disc_get_metrics": (_st, [_vp, _i32, _f32, _f32, _f32, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]),
    "disc_k_force_update": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32,
                                  ctypes.POINTER(_i32), _f32, _f32, _i32, _vp]),
    "disc_k_ssd_loss": (_st, [_vp, _vp, _vp, _vp, _i32, _i32, _i32, ctypes.POINTER(_i32), _f32, _f32, _vp]),
    "disc_k_ssd_grad": (_st, [_vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32, ctypes.POINTER(_i32), _f32, _f32,
                              _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def header_functions(path=HEADER):
    """Names of the functions include/disc.h declares."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:disc_status|float|const char\*)\s+(disc_\w+)\s*\(", src, re.M)))


def _check(status, where):
    if status != 0:
        raise DiscError(status, where)


def bounds_violations(stream=None):
    """(out-of-range accesses counted since the last call, whether this is the
    bounds-checked build): disc_bounds_violations."""
    n, chk = _i64(0), _i32(0)
    _check(_lib.disc_bounds_violations(_stream(stream), ctypes.byref(n), ctypes.byref(chk)),
           "disc_bounds_violations")
    return int(n.value), bool(chk.value)


SW_NO_TMA, SW_TMA_STALL, SW_NO_GRAPH, SW_UNROLLED_GRAPH, SW_FAULT_ALLOC, SW_WIDE_ANY = 1, 2, 4, 8, 16, 32
SW_SEPARATE_WARP, SW_FUSED_WARP = 64, 128


class test_switches:
    """Context manager: set the library's test switches (disc_set_test_switches)
    to `flags` inside the block and restore the previous ones after it."""
    __test__ = False

    def __init__(self, flags):
        self.flags = int(flags)

    def __enter__(self):
        old = ctypes.c_uint32(0)
        _check(_lib.disc_set_test_switches(self.flags, ctypes.byref(old)), "disc_set_test_switches")
        self.old = old.value
        return self

    def __exit__(self, *exc):
        _check(_lib.disc_set_test_switches(self.old, None), "disc_set_test_switches")


def _ptr(t):
    """Raw pointer of a torch tensor (device) or numpy array (host)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffer must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _mem_kind(t):
    if isinstance(t, np.ndarray):
        return MEM_HOST
    return MEM_DEVICE if t.is_cuda else MEM_HOST


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _f32_check(t, shape, name):
    if isinstance(t, np.ndarray):
        if t.dtype != np.float32:
            raise TypeError(f"{name} must be float32")
    else:
        import torch
        if t.dtype != torch.float32:
            raise TypeError(f"{name} must be float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def make_params(patch=(3, 3, 3), sigma=1.0, radius=0, levels=2, iters=(50, 50), stop_eps=0.0,
                stop_window=10, force_mode=FORCE_THIRION, global_shift=True, var_floor=1e-6,
                mask_mode=0, hu0_factor=2.0, a_lo=0.5, a_hi=1.5, fill_h=50.0, fill_t=(7, 7, 3),
                fill_passes=32, smooth_mode=0, quant_max=(0.0, 0.0), norm_planes=(0, 0)):
    p = Params()
    _check(_lib.disc_params_default(ctypes.byref(p)), "disc_params_default")
    for a in range(3):
        p.patch[a] = int(patch[a])
    p.gauss_sigma = float(sigma)
    p.gauss_radius = int(radius)
    p.levels = int(levels)
    iters = list(iters)
    if len(iters) != levels:
        raise ValueError("one iteration count per level (coarsest first)")
    for i in range(MAX_LEVELS):
        p.iters[i] = int(iters[i]) if i < len(iters) else 0
    p.stop_eps = float(stop_eps)
    p.stop_window = int(stop_window)
    p.force_mode = int(force_mode)
    p.global_shift = 1 if global_shift else 0
    p.var_floor = float(var_floor)
    p.mask_mode = int(mask_mode)
    p.hu0_factor = float(hu0_factor)
    p.a_lo = float(a_lo)
    p.a_hi = float(a_hi)
    p.fill_h = float(fill_h)
    for a in range(3):
        p.fill_t[a] = int(fill_t[a])
    p.fill_passes = int(fill_passes)
    p.smooth_mode = int(smooth_mode)
    p.quant_max[0] = float(quant_max[0])
    p.quant_max[1] = float(quant_max[1])
    p.norm_planes[0] = int(norm_planes[0])
    p.norm_planes[1] = int(norm_planes[1])
    return p


class Registration:
    """One DISC registration context (disc_create .. disc_destroy).

    ``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None for the
    current torch stream.
    """

    def __init__(self, params: Params | None = None, device=0, stream=None, **kw):
        if params is None:
            params = make_params(**kw)
        self.params = params
        self.device = device
        self._stream = _stream(stream)
        h = _vp()
        _check(_lib.disc_create(ctypes.byref(params), device, self._stream, ctypes.byref(h)), "disc_create")
        self._h = h
        self.dims = None

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.disc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls ---------------------------------------------------------------
    def set_images(self, ct, cbct):
        nz, ny, nx = ct.shape
        _f32_check(ct, (nz, ny, nx), "ct")
        _f32_check(cbct, (nz, ny, nx), "cbct")
        kind = _mem_kind(ct)
        if _mem_kind(cbct) != kind:
            raise ValueError("ct and cbct must both be host or both be device buffers")
        _check(_lib.disc_set_images(self._h, _ptr(ct), _ptr(cbct), nx, ny, nz, kind), "disc_set_images")
        self.dims = (nx, ny, nz)

    def iterate(self, max_iters=-1, sync=True):
        if sync:
            done, last = _i32(0), _f32(0)
            _check(_lib.disc_iterate(self._h, int(max_iters), ctypes.byref(done), ctypes.byref(last)),
                   "disc_iterate")
            return int(done.value), float(last.value)
        _check(_lib.disc_iterate(self._h, int(max_iters), None, None), "disc_iterate")
        return None

    def get_field(self, out=None):
        nx, ny, nz = self.dims
        if out is None:
            out = np.empty((3, nz, ny, nx), np.float32)
        _f32_check(out, (3, nz, ny, nx), "out")
        _check(_lib.disc_get_field(self._h, _ptr(out), _mem_kind(out)), "disc_get_field")
        return out

    def progress(self):
        lev, it = _i32(0), _i32(0)
        dims = (_i32 * 3)()
        _check(_lib.disc_get_progress(self._h, ctypes.byref(lev), ctypes.byref(it), dims), "disc_get_progress")
        return int(lev.value), int(it.value), (dims[0], dims[1], dims[2])

    def get_corrected(self, out=None):
        _, _, (nx, ny, nz) = self.progress()
        if out is None:
            out = np.empty((nz, ny, nx), np.float32)
        _f32_check(out, (nz, ny, nx), "out")
        _check(_lib.disc_get_corrected(self._h, _ptr(out), _mem_kind(out)), "disc_get_corrected")
        return out

    def get_level_field(self, level, out):
        """Level `level`'s own field ([3][nz][ny][nx] of that level, its voxel units) into `out`."""
        _check(_lib.disc_get_level_field(self._h, int(level), _ptr(out), _mem_kind(out)), "disc_get_level_field")
        return out

    def set_field(self, level, r):
        _check(_lib.disc_set_field(self._h, int(level), _ptr(r), _mem_kind(r)), "disc_set_field")

    def norm_history(self, level, cap=100000):
        out = np.empty(cap, np.float32)
        n = _i32(0)
        _check(_lib.disc_get_norm_history(self._h, int(level), out.ctypes.data, cap, ctypes.byref(n)),
               "disc_get_norm_history")
        return out[:n.value].copy()

    def norm_sums(self, level, cap=100000):
        """[k][2]: sum |dr|, sum |r| behind each l^(k) of `level` (float64)."""
        out = np.empty((cap, 2), np.float64)
        n = _i32(0)
        _check(_lib.disc_get_norm_sums(self._h, int(level), out.ctypes.data, cap, ctypes.byref(n)),
               "disc_get_norm_sums")
        return out[:n.value].copy()

    def metrics(self, bins=64, sigma=1.0, t_low=0.4, t_high=0.2):
        """(NMI, edge RMSE of Eq. 11) between I_m(x + r(x)) and I'_s at the current level."""
        nmi, rmse = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(_lib.disc_get_metrics(self._h, int(bins), float(sigma), float(t_low), float(t_high),
                                     ctypes.byref(nmi), ctypes.byref(rmse)), "disc_get_metrics")
        return nmi.value, rmse.value

    def ssd(self, level, r, grad=None):
        """SSD loss of field r on pyramid level `level` (disc_ssd); with `grad` (same
        kind and shape as r) also dL/dr.  Returns the loss."""
        loss = ctypes.c_double(0.0)
        kind = _mem_kind(r)
        if grad is not None and _mem_kind(grad) != kind:
            raise ValueError("r and grad must both be host or both be device buffers")
        _check(_lib.disc_ssd(self._h, int(level), _ptr(r), ctypes.byref(loss),
                             _ptr(grad) if grad is not None else None, kind), "disc_ssd")
        return loss.value

    def correction_means(self):
        """(mean a, mean b, voxels) of Eqs. 5-6 for the current field and level (disc_get_correction_means)."""
        ma, mb, n = ctypes.c_double(0.0), ctypes.c_double(0.0), _i64(0)
        _check(_lib.disc_get_correction_means(self._h, ctypes.byref(ma), ctypes.byref(mb), ctypes.byref(n)),
               "disc_get_correction_means")
        return ma.value, mb.value, int(n.value)

    def launch_count(self):
        """Kernel launches disc_iterate has issued on this context (disc_get_launch_count)."""
        n = _i64(0)
        _check(_lib.disc_get_launch_count(self._h, ctypes.byref(n)), "disc_get_launch_count")
        return int(n.value)

    def mask_constants(self):
        """(HU0, a_m) fixed at set_images when the mask is on (Eq. 7, Sec. 2.3)."""
        hu0, am = _f32(0.0), _f32(0.0)
        _check(_lib.disc_get_mask_constants(self._h, ctypes.byref(hu0), ctypes.byref(am)),
               "disc_get_mask_constants")
        return hu0.value, am.value


class Batch:
    """Many pairs advanced together (disc_batch_create .. disc_batch_destroy)."""

    def __init__(self, npairs, params: Params | None = None, device=0, stream=None, **kw):
        if params is None:
            params = make_params(**kw)
        self.params = params
        self.npairs = int(npairs)
        h = _vp()
        _check(_lib.disc_batch_create(ctypes.byref(params), device, _stream(stream), self.npairs,
                                      ctypes.byref(h)), "disc_batch_create")
        self._h = h
        self.dims = [None] * self.npairs

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.disc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_images(self, pair, ct, cbct):
        nz, ny, nx = ct.shape
        _f32_check(ct, (nz, ny, nx), "ct")
        _f32_check(cbct, (nz, ny, nx), "cbct")
        kind = _mem_kind(ct)
        _check(_lib.disc_batch_set_images(self._h, int(pair), _ptr(ct), _ptr(cbct), nx, ny, nz, kind),
               "disc_batch_set_images")
        self.dims[pair] = (nx, ny, nz)

    def restart(self):
        _check(_lib.disc_batch_restart(self._h), "disc_batch_restart")

    def iterate(self, max_iters=-1):
        done = _i32(0)
        _check(_lib.disc_batch_iterate(self._h, int(max_iters), ctypes.byref(done)), "disc_batch_iterate")
        return int(done.value)

    def get_field(self, pair, out=None):
        nx, ny, nz = self.dims[pair]
        if out is None:
            out = np.empty((3, nz, ny, nx), np.float32)
        _f32_check(out, (3, nz, ny, nx), "out")
        _check(_lib.disc_batch_get_field(self._h, int(pair), _ptr(out), _mem_kind(out)), "disc_batch_get_field")
        return out

    def tuning(self, level):
        items, grid, zmult = _i32(0), _i32(0), _i32(0)
        _check(_lib.disc_batch_get_tuning(self._h, int(level), ctypes.byref(items), ctypes.byref(grid),
                                          ctypes.byref(zmult)), "disc_batch_get_tuning")
        return int(items.value), int(grid.value), int(zmult.value)

    def box_path(self, level):
        """`level`'s moment/force kernel: 2 wide tiles, 1 bulk-copy-fed 32 x 16, 0 per-thread loads."""
        t = _i32(0)
        _check(_lib.disc_batch_get_box_path(self._h, int(level), ctypes.byref(t)), "disc_batch_get_box_path")
        return int(t.value)

    def box_path_tma(self, level):
        """True when `level`'s moment/force launch is the bulk-tensor-copy-fed 32 x 16 kernel."""
        return self.box_path(level) == 1

    def gauss_tuning(self, level):
        """(z chunk of the Gaussian z pass, 0 = pair plans; 1 if the warp runs after the Gaussian) at `level`."""
        zlen, sep = _i32(0), _i32(0)
        _check(_lib.disc_batch_get_gauss_tuning(self._h, int(level), ctypes.byref(zlen), ctypes.byref(sep)),
               "disc_batch_get_gauss_tuning")
        return int(zlen.value), int(sep.value)

    def pin_tuning(self, level, zmult, grid):
        """Use z chunking `zmult` and grid `grid` (0: one CTA per item) at `level` instead of the autotuner."""
        _check(_lib.disc_batch_pin_tuning(self._h, int(level), int(zmult), int(grid)), "disc_batch_pin_tuning")


def norm_stop_rule(sums, window, eps):
    """Sec. 2.3 on summed norms (disc_norm_stop_rule): `sums` [k][2] float64 (sum |dr|,
    sum |r| per iteration of a level).  Returns (l history float32, stop after the last)."""
    s = np.ascontiguousarray(sums, np.float64).reshape(-1, 2)
    l_out = np.empty(s.shape[0], np.float32)
    stop = _i32(0)
    _check(_lib.disc_norm_stop_rule(s.ctypes.data, s.shape[0], int(window), float(eps), l_out.ctypes.data,
                                    ctypes.byref(stop)), "disc_norm_stop_rule")
    return l_out, bool(stop.value)


# ---------------------------------------------------------------------------
# Kernel-level calls (device tensors, caller's stream)
# ---------------------------------------------------------------------------

def qscale(max_abs, patch):
    p = (_i32 * 3)(*patch)
    return float(_lib.disc_qscale(float(max_abs), p))


def k_max_abs(v, out, stream=None):
    _check(_lib.disc_k_max_abs(_ptr(v), v.numel(), _ptr(out), _stream(stream)), "disc_k_max_abs")


def k_global_shift(Im, Is, Is_out, delta_out=None, stream=None):
    _check(_lib.disc_k_global_shift(_ptr(Im), _ptr(Is), _ptr(Is_out), Im.numel(), _ptr(delta_out),
                                    _stream(stream)), "disc_k_global_shift")


def k_downsample2(inp, out, stream=None):
    nz, ny, nx = inp.shape
    _check(_lib.disc_k_downsample2(_ptr(inp), _ptr(out), nx, ny, nz, _stream(stream)), "disc_k_downsample2")


def k_upsample_field2(rc, rf, stream=None):
    _, nz, ny, nx = rf.shape
    _check(_lib.disc_k_upsample_field2(_ptr(rc), _ptr(rf), nx, ny, nz, _stream(stream)),
           "disc_k_upsample_field2")


def k_static_norm(Is, zs, patch, qs, var_floor=1e-6, stream=None):
    nz, ny, nx = Is.shape
    p = (_i32 * 3)(*patch)
    _check(_lib.disc_k_static_norm(_ptr(Is), _ptr(zs), nx, ny, nz, p, float(qs), float(var_floor),
                                   _stream(stream)), "disc_k_static_norm")


def k_warp(Im, r, m, stream=None):
    nz, ny, nx = Im.shape
    _check(_lib.disc_k_warp(_ptr(Im), _ptr(r), _ptr(m), nx, ny, nz, _stream(stream)), "disc_k_warp")


def k_pass_a(Im, zs, r, u, patch, qs, m_out=None, d_out=None, norms_out=None, var_floor=1e-6,
             force_mode=FORCE_THIRION, stream=None):
    """Warp, patch moments, correction, force and update; d_out gets I'_s - m."""
    nz, ny, nx = Im.shape
    p = (_i32 * 3)(*patch)
    _check(_lib.disc_k_pass_a(_ptr(Im), _ptr(zs), _ptr(r), _ptr(u), _ptr(m_out), _ptr(d_out),
                              _ptr(norms_out), nx, ny, nz, p, float(qs), float(var_floor),
                              int(force_mode), _stream(stream)), "disc_k_pass_a")


def k_pass_a_static(Im, zs, r, u, m_out, patch, qs, d_out=None, norms_out=None, var_floor=1e-6,
                    force_mode=FORCE_THIRION, stream=None):
    """disc_k_pass_a without device allocation (fixed in-library scratch; m_out required)."""
    nz, ny, nx = Im.shape
    p = (_i32 * 3)(*patch)
    _check(_lib.disc_k_pass_a_static(_ptr(Im), _ptr(zs), _ptr(r), _ptr(u), _ptr(m_out), _ptr(d_out),
                                     _ptr(norms_out), nx, ny, nz, p, float(qs), float(var_floor),
                                     int(force_mode), _stream(stream)), "disc_k_pass_a_static")


def k_gauss(u, r, sigma, radius=0, stream=None):
    _, nz, ny, nx = u.shape
    _check(_lib.disc_k_gauss(_ptr(u), _ptr(r), nx, ny, nz, float(sigma), int(radius), _stream(stream)),
           "disc_k_gauss")


def k_static_stats(Is, zs, sd, patch, qs, var_floor=1e-6, stream=None):
    """CBCT normalisation zs and STD(S) per voxel (sd may be None)."""
    nz, ny, nx = Is.shape
    p = (_i32 * 3)(*patch)
    _check(_lib.disc_k_static_stats(_ptr(Is), _ptr(zs), _ptr(sd), nx, ny, nz, p, float(qs), float(var_floor),
                                    _stream(stream)), "disc_k_static_stats")


def k_ratio_median(m, zs, sd, a_work, median_out, patch, qs, var_floor=1e-6, stream=None):
    """a = STD(M)/STD(S) into a_work (-1 where undefined) and its median (device double)."""
    nz, ny, nx = m.shape
    p = (_i32 * 3)(*patch)
    _check(_lib.disc_k_ratio_median(_ptr(m), _ptr(zs), _ptr(sd), _ptr(a_work), _ptr(median_out), nx, ny, nz, p,
                                    float(qs), float(var_floor), _stream(stream)), "disc_k_ratio_median")


def k_correct_masked(m, Is, zs, sd, a, b, d, stamp, patch, qs, hu0, a_min, a_max, fill_h=50.0,
                     fill_t=(7, 7, 3), fill_passes=32, remaining_out=None, var_floor=1e-6, stream=None):
    """Mask (Eq. 7) and fill (Eqs. 8-10) of one correction; d = I'_s - m, stamp int32."""
    nz, ny, nx = m.shape
    p = (_i32 * 3)(*patch)
    t = (_i32 * 3)(*fill_t)
    _check(_lib.disc_k_correct_masked(_ptr(m), _ptr(Is), _ptr(zs), _ptr(sd), _ptr(a), _ptr(b), _ptr(d),
                                      _ptr(stamp), _ptr(remaining_out), nx, ny, nz, p, float(qs),
                                      float(var_floor), float(hu0), float(a_min), float(a_max), float(fill_h),
                                      t, int(fill_passes), _stream(stream)), "disc_k_correct_masked")


def k_force(m, d, r, u, norms_out=None, force_mode=FORCE_THIRION, stream=None):
    """Demons force and update from d = I'_s - m and m."""
    nz, ny, nx = m.shape
    _check(_lib.disc_k_force(_ptr(m), _ptr(d), _ptr(r), _ptr(u), _ptr(norms_out), nx, ny, nz, int(force_mode),
                             _stream(stream)), "disc_k_force")


def k_nmi(a, b, out, bins=64, stream=None):
    """Normalised mutual information of two images into out (device double)."""
    _check(_lib.disc_k_nmi(_ptr(a), _ptr(b), int(a.numel()), int(bins), _ptr(out), _stream(stream)), "disc_k_nmi")


def k_canny(img, edges, sigma=1.0, t_low=0.4, t_high=0.2, stream=None):
    """Binary Canny edges (uint8 tensor like img), slice by slice."""
    nz, ny, nx = img.shape
    _check(_lib.disc_k_canny(_ptr(img), _ptr(edges), nx, ny, nz, float(sigma), float(t_low), float(t_high),
                             _stream(stream)), "disc_k_canny")


def k_edge_rmse(e1, e2, out, stream=None):
    """Eq. (11) of two binary edge images into out (device double)."""
    _check(_lib.disc_k_edge_rmse(_ptr(e1), _ptr(e2), int(e1.numel()), _ptr(out), _stream(stream)),
           "disc_k_edge_rmse")


def k_check_error(stream=None):
    """Synchronise the stream; raise DiscError if a bounded device wait gave up."""
    _check(_lib.disc_k_check_error(_stream(stream)), "disc_k_check_error")


def k_force_update(m, zs, r, u, patch, qs, d_out=None, norms_out=None, var_floor=1e-6,
                   force_mode=FORCE_THIRION, stream=None):
    """Moment, correction, force and update pass on a given warped image m."""
    nz, ny, nx = m.shape
    p = (_i32 * 3)(*patch)
    _check(_lib.disc_k_force_update(_ptr(m), _ptr(zs), _ptr(r), _ptr(u), _ptr(d_out), _ptr(norms_out),
                                    nx, ny, nz, p, float(qs), float(var_floor), int(force_mode),
                                    _stream(stream)), "disc_k_force_update")


def k_ssd_loss(Im, zs, r, loss_out, patch, qs, var_floor=1e-6, stream=None):
    nz, ny, nx = Im.shape
    p = (_i32 * 3)(*patch)
    _check(_lib.disc_k_ssd_loss(_ptr(Im), _ptr(zs), _ptr(r), _ptr(loss_out), nx, ny, nz, p, float(qs),
                                float(var_floor), _stream(stream)), "disc_k_ssd_loss")


def k_ssd_grad(Im, zs, r, grad, patch, qs, loss_out=None, var_floor=1e-6, stream=None):
    nz, ny, nx = Im.shape
    p = (_i32 * 3)(*patch)
    _check(_lib.disc_k_ssd_grad(_ptr(Im), _ptr(zs), _ptr(r), _ptr(grad), _ptr(loss_out), nx, ny, nz, p,
                                float(qs), float(var_floor), _stream(stream)), "disc_k_ssd_grad")
