"""The bounds-checked build (libdisc_bc.so, compiled with -DDISC_BOUNDS_CHECK):
the memory-safety check of the per-iteration kernels, in place of a sanitizer.

In that build every global index of the warp, the moment/force passes (the
32 x 16 tilings with and without bulk tensor copies, and the wide-tile pass),
the Gaussian passes and the pyramid up- and down-sampling is tested against
its buffer's extent before the access; an index out of range is counted on
the device, never trapped.  A child process loads the checked build
(DISC_LIBRARY=bounds) and runs the small parity cases of the kernel and
registration tests; no access may be out of range, and every output must be
the normal build's bit for bit (the checks change no arithmetic).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_cases():
    """Outputs of the small parity cases through whichever library `disc` loaded."""
    import torch
    from paper_1204_6295_b300 import disc, phantom
    from gpu_util import ct_like, dev, empty, host
    out = {}
    cases = [((13, 37, 70), 3, 0), ((24, 52, 64), 11, 0), ((21, 45, 70), 5, 0), ((33, 64, 96), 5, disc.SW_WIDE_ANY),
             ((9, 33, 35), 15, 0), ((2, 17, 1), 5, 0)]
    for i, (shape, p, sw) in enumerate(cases):
        P = (p, p, p)
        Im = ct_like(shape, 10 + i)
        Is = ct_like(shape, 20 + i, noise=25.0)
        r = (phantom.smooth_random_field(shape, 30 + i, amp=2.0) if min(shape) > 1
             else phantom.random_field(shape, 30 + i, amp=1.5))
        qs_s = disc.qscale(float(np.abs(Is).max()), P)
        qs_m = disc.qscale(float(np.abs(Im).max()), P)
        with disc.test_switches(sw):
            zs = empty(*shape)
            disc.k_static_norm(dev(Is), zs, P, qs_s)
            u, m, d = empty(3, *shape), empty(*shape), empty(*shape)
            norms = torch.zeros(2, dtype=torch.float64, device="cuda")
            disc.k_pass_a(dev(Im), zs, dev(r), u, P, qs_m, m_out=m, d_out=d, norms_out=norms)
            g = empty(3, *shape)
            disc.k_gauss(u, g, 1.5)
        for name, t in (("zs", zs), ("u", u), ("m", m), ("d", d), ("norms", norms), ("g", g)):
            out[f"{name}{i}"] = host(t)
    # pyramid
    f = dev(phantom.smooth_random_field((17, 30, 26), 41, amp=2.0))
    c = empty(3, 9, 15, 13)
    for k in range(3):
        disc.k_downsample2(f[k], c[k])
    up = empty(3, 17, 30, 26)
    disc.k_upsample_field2(c, up)
    out["down"], out["up"] = host(c), host(up)
    # registrations: two levels, Thirion and double force, and a batch of two pairs
    pair = phantom.ellipsoid_pair(48, 40, 24, seed=43)
    for fm in (0, 1):
        with disc.Registration(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(4, 3), force_mode=fm) as reg:
            reg.set_images(pair.ct, pair.cbct)
            reg.iterate(-1)
            out[f"reg{fm}"] = reg.get_field()
    pairs = [phantom.ellipsoid_pair(40, 32, 20, seed=44), phantom.ellipsoid_pair(96, 64, 24, seed=45)]
    with disc.Batch(2, patch=(5, 5, 5), sigma=1.0, levels=2, iters=(3, 3)) as b:
        for k, p in enumerate(pairs):
            b.set_images(k, p.ct, p.cbct)
        b.iterate(-1)
        for k in range(2):
            out[f"batch{k}"] = b.get_field(k)
    torch.cuda.synchronize()
    return out


def test_bounds_checked_build_runs_clean_and_matches(tmp_path):
    lib = os.path.join(ROOT, "paper_1204_6295_b300", "libdisc_bc.so")
    assert os.path.exists(lib), "the bounds-checked build is made by __graft_entry__.build()"
    npz = str(tmp_path / "bounds.npz")
    code = (
        "import sys, numpy as np\n"
        f"sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'tests')!r})\n"
        "import test_gpu_bounds as T\n"
        "from paper_1204_6295_b300 import disc\n"
        "assert disc.LIB_PATH.endswith('libdisc_bc.so')\n"
        "disc.bounds_violations()                    # clear\n"
        "out = T.run_cases()\n"
        "n, checked = disc.bounds_violations()\n"
        f"np.savez({npz!r}, violations=n, checked=checked, **out)\n"
    )
    env = dict(os.environ, DISC_LIBRARY="bounds")
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    got = np.load(npz)
    assert bool(got["checked"]), "the child did not load the bounds-checked build"
    assert int(got["violations"]) == 0, int(got["violations"])
    from paper_1204_6295_b300 import disc
    n, checked = disc.bounds_violations()
    assert not checked and n == 0                  # this process runs the normal build
    ref = run_cases()
    for k, v in ref.items():
        np.testing.assert_array_equal(got[k], v, err_msg=k)
