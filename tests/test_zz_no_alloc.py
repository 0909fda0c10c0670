"""The allocation-free entry point disc_k_pass_a_static.

It serves callers that cannot let the library allocate device memory (an
application that owns all device memory through its own pool or a fixed
budget, or a host that forbids plug-ins from allocating).  Its only scratch is
a fixed array inside the library that every call reuses.  On the volumes of
this test it runs the same kernels with the same launch plan as the
allocating entry point disc_k_pass_a, so this test calls both through the C
ABI, twice in a row on
inputs of different sizes (the larger grid first, so that the second call
would read partial sums the first one left behind if it read any it did not
write), and requires bitwise equal m, d, u and norms.  Each result is also
checked against the FP64 oracle's force on the GPU's own m and d, within the
per-kernel tolerance of the other parity tests.  The file name makes pytest
collect it last.
"""
import ctypes

import numpy as np
import pytest

from oracle import disc_oracle as O
from paper_1204_6295_b300 import phantom

from gpu_util import ct_like, dev, empty, host

pytestmark = pytest.mark.gpu

TOL = 1e-5

# (nz, ny, nx), patch: the first launch has more CTAs than the second
CALLS = [((21, 45, 70), (5, 5, 5), 33), ((13, 18, 36), (3, 3, 3), 34)]


def test_static_scratch_pass_a_equals_allocating_entry_point_bitwise_twice():
    import torch
    from paper_1204_6295_b300 import disc
    for call, (shape, patch, seed) in enumerate(CALLS):
        Im = ct_like(shape, seed)
        Is = ct_like(shape, seed + 100, noise=25.0)
        qs_s = disc.qscale(float(np.abs(Is).max()), patch)
        qs_m = disc.qscale(float(np.abs(Im).max()), patch)
        zs = empty(*shape)
        disc.k_static_norm(dev(Is), zs, patch, qs_s)
        Im_d = dev(Im)
        r_np = phantom.smooth_random_field(shape, seed, amp=2.0)
        r = dev(r_np)
        u_ref, m_ref, d_ref = empty(3, *shape), empty(*shape), empty(*shape)
        n_ref = torch.zeros(2, dtype=torch.float64, device="cuda")
        disc.k_pass_a(Im_d, zs, r, u_ref, patch, qs_m, m_out=m_ref, d_out=d_ref, norms_out=n_ref)
        u, m, d = empty(3, *shape), empty(*shape), empty(*shape)
        norms = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        p = (ctypes.c_int32 * 3)(*patch)
        status = disc._lib.disc_k_pass_a_static(
            Im_d.data_ptr(), zs.data_ptr(), r.data_ptr(), u.data_ptr(), m.data_ptr(), d.data_ptr(),
            norms.data_ptr(), shape[2], shape[1], shape[0], p, qs_m, 1e-6, 0,
            torch.cuda.current_stream().cuda_stream)
        assert status == 0, (call, disc._lib.disc_status_str(status))
        # the same kernels on the same inputs: bit for bit
        np.testing.assert_array_equal(host(m), host(m_ref), err_msg=f"m, call {call}")
        np.testing.assert_array_equal(host(d), host(d_ref), err_msg=f"d, call {call}")
        np.testing.assert_array_equal(host(u), host(u_ref), err_msg=f"u, call {call}")
        np.testing.assert_array_equal(host(norms), host(n_ref), err_msg=f"norms, call {call}")
        # and the force against the oracle's (Eq. 1) on the GPU's own m and I'_s = m + d
        m_g, f_g = host(m), host(m) + host(d)
        dr_ref = O.force(m_g, f_g, O.FORCE_THIRION)
        dr_g = host(u) - r_np.astype(np.float64)
        scale = max(np.abs(dr_ref).max(), 1e-3)
        assert np.abs(dr_g - dr_ref).max() <= TOL * scale, call
        n_g = host(norms)
        assert n_g[0] == pytest.approx(np.sqrt((dr_ref ** 2).sum(0)).sum(), rel=1e-5, abs=1e-6)
        assert n_g[1] == pytest.approx(np.sqrt((r_np.astype(np.float64) ** 2).sum(0)).sum(), rel=1e-5)


def test_static_scratch_pass_a_rejects_grids_beyond_its_scratch():
    """Launches larger than the fixed scratch are refused before any work is
    queued.  The buffers are real device memory of the right sizes, so that a
    call that did run would only compute on them."""
    import torch
    from paper_1204_6295_b300 import disc
    p = (ctypes.c_int32 * 3)(3, 3, 3)
    # a 4096 x 4096 plane needs 128 x 256 tiles of 32 x 16: more CTAs than the fixed scratch holds
    shape = (1, 4096, 4096)
    Im, zs, m = empty(*shape), empty(*shape), empty(*shape)
    r, u = empty(3, *shape), empty(3, *shape)
    for t in (Im, zs, m, r):
        t.zero_()
    status = disc._lib.disc_k_pass_a_static(Im.data_ptr(), zs.data_ptr(), r.data_ptr(), u.data_ptr(),
                                            m.data_ptr(), None, None, 4096, 4096, 1, p, 1.0, 1e-6, 0,
                                            torch.cuda.current_stream().cuda_stream)
    assert status == 2
    small = (8, 8, 8)
    Im, zs, r, u = empty(*small), empty(*small), empty(3, *small), empty(3, *small)
    assert disc._lib.disc_k_pass_a_static(Im.data_ptr(), zs.data_ptr(), r.data_ptr(), u.data_ptr(), None, None,
                                          None, 8, 8, 8, p, 1.0, 1e-6, 0, None) == 1     # m_out is required
    torch.cuda.synchronize()
