"""The allocation-free entry point disc_k_pass_a_static.

It serves callers that cannot let the library allocate device memory (an
application that owns all device memory through its own pool or a fixed
budget, or a host that forbids plug-ins from allocating).  Its only scratch is
a fixed array inside the library that every call reuses, so this test calls it
twice in a row through the C ABI and checks both results against the
allocating entry point disc_k_pass_a, within the per-kernel tolerance used by
the other parity tests.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, empty, host, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_static_scratch_pass_a_matches_allocating_entry_point_twice():
    import torch
    from paper_1204_6295_b300 import disc
    shape, patch = (21, 45, 70), (5, 5, 5)
    Im = ct_like(shape, 31)
    Is = ct_like(shape, 32, noise=25.0)
    qs_s = disc.qscale(float(np.abs(Is).max()), patch)
    qs_m = disc.qscale(float(np.abs(Im).max()), patch)
    zs = empty(*shape)
    disc.k_static_norm(dev(Is), zs, patch, qs_s)
    Im_d = dev(Im)
    u_ref, m_ref, d_ref = empty(3, *shape), empty(*shape), empty(*shape)
    n_ref = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call, seed in enumerate((33, 34)):
        r = dev(phantom.smooth_random_field(shape, seed, amp=2.0))
        disc.k_pass_a(Im_d, zs, r, u_ref, patch, qs_m, m_out=m_ref, d_out=d_ref, norms_out=n_ref)
        u, m, d = empty(3, *shape), empty(*shape), empty(*shape)
        norms = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        p = (ctypes.c_int32 * 3)(*patch)
        status = disc._lib.disc_k_pass_a_static(
            Im_d.data_ptr(), zs.data_ptr(), r.data_ptr(), u.data_ptr(), m.data_ptr(), d.data_ptr(),
            norms.data_ptr(), shape[2], shape[1], shape[0], p, qs_m, 1e-6, 0,
            torch.cuda.current_stream().cuda_stream)
        assert status == 0, (call, disc._lib.disc_status_str(status))
        assert rel_err(host(m), host(m_ref)) <= TOL, call
        assert rel_err(host(d), host(d_ref)) <= TOL, call
        assert rel_err(host(u) - host(r), host(u_ref) - host(r)) <= TOL, call
        np.testing.assert_allclose(host(norms), host(n_ref), rtol=TOL)


def test_static_scratch_pass_a_rejects_grids_beyond_its_scratch():
    import torch
    from paper_1204_6295_b300 import disc
    p = (ctypes.c_int32 * 3)(3, 3, 3)
    fake = ctypes.c_void_p(256)
    other = ctypes.c_void_p(512)
    # a 4096 x 4096 plane needs 128 x 256 tiles: more CTAs than the fixed scratch holds
    status = disc._lib.disc_k_pass_a_static(fake, fake, fake, other, fake, None, None, 4096, 4096, 1, p,
                                            1.0, 1e-6, 0, torch.cuda.current_stream().cuda_stream)
    assert status == 2
    assert disc._lib.disc_k_pass_a_static(fake, fake, fake, other, None, None, None, 8, 8, 8, p, 1.0, 1e-6,
                                          0, None) == 1     # m_out is required
