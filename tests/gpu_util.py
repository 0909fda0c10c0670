"""Helpers shared by the GPU tests: device transfers and tolerance checks."""
import numpy as np


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def empty(*shape):
    import torch
    return torch.empty(*shape, dtype=torch.float32, device="cuda")


def rel_err(got, ref):
    """max |got - ref| / max |ref| (the per-kernel norm of the parity bar)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.abs(ref).max()
    if scale == 0:
        return np.abs(got).max()
    return np.abs(got - ref).max() / scale


def ct_like(shape, seed, noise=0.0):
    """Piecewise-smooth CT-like volume: smooth blobs plus two sharp levels (HU range)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = np.zeros(shape)
    for _ in range(5):
        k = rng.uniform(0.05, 0.5, size=3)
        v += rng.uniform(50, 250) * np.sin(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, 6))
    cx, cy, cz = nx / 2, ny / 2, nz / 2
    s = ((x - cx) / max(nx / 3, 1)) ** 2 + ((y - cy) / max(ny / 3, 1)) ** 2 + ((z - cz) / max(nz / 3, 1)) ** 2
    v += np.where(s < 1.0, 600.0, -400.0)
    if noise > 0:
        v += rng.normal(0, noise, size=shape)
    return v.astype(np.float32)
