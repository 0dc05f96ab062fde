"""The allocation-free entry point lbm_global_balance_static, called through
the C ABI with ctypes, against lbm_global_balance on the same states.

It serves callers that cannot allocate device memory (for instance a plug-in
whose host application owns the device memory pool), so it takes no
workspace and keeps its scratch in a fixed device array.  Two calls in a row
on different states must each match the handle-based entry point within the
tolerance the other global-balance tests use (1e-12 relative; the momentum
sums, which cancel, to 1e-12 per cell), and so must one call against the
FP64 oracle directly.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    lib = P.load_library()
    lib.lbm_global_balance_static.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(P._MemberCfg), ctypes.c_void_p,
                                              ctypes.c_void_p]
    lib.lbm_global_balance_static.restype = ctypes.c_int
    lib.lbm_static_last_error.restype = ctypes.c_char_p
    return P


def _static_call(P, f_dev, member, stream):
    lib = P.load_library()
    out = np.full(P.NGLOBAL, np.nan)
    cfg = member.c()
    rc = lib.lbm_global_balance_static(ctypes.c_void_p(f_dev.data_ptr()), member.nx, member.ny,
                                       ctypes.byref(cfg), out.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.lbm_static_last_error().decode()
    return out


def _compare(got, ref, ncell):
    np.testing.assert_allclose(got[[0, 3, 4, 5, 6]], ref[[0, 3, 4, 5, 6]], rtol=1e-12)
    assert abs(got[1] - ref[1]) < 1e-12 * ncell and abs(got[2] - ref[2]) < 1e-12 * ncell


def test_static_matches_handle_entry_point_twice(P):
    import torch
    nx, ny, tau = 96, 80, 0.57
    m = P.Member(nx, ny, tau, 1.0, 1, 3, 2e-4, 1e-3)
    lat = P.Lattice([m], precision=64)
    stream = torch.cuda.current_stream()
    for seed in (11, 12):  # two calls in a row, on different states
        f = li.random_populations(nx, ny, seed=seed, rel_noise=0.03)
        lat.set_populations(0, f)
        ref = lat.global_balance(0)
        f_dev = lat.get_populations(0)
        got = _static_call(P, f_dev, m, stream)
        _compare(got, ref, nx * ny)


def test_static_at_the_size_limit_and_unforced(P):
    import torch
    n = 512  # LBM_STATIC_MAX_CELLS = 512 * 512
    m = P.Member(n, n, 0.52)
    lat = P.Lattice([m], precision=32)
    lat.init_fields(0, *li.random_phase(n, seed=3, u_rms=0.02))
    lat.step(5)
    ref = lat.global_balance(0)
    got = _static_call(P, lat.get_populations(0), m, torch.cuda.current_stream())
    _compare(got, ref, n * n)


def test_static_matches_the_oracle_after_a_size_change(P, orc):
    """The whole-grid quantities straight against the FP64 oracle, and a
    grid shrinking between calls: a 512^2 call, then 5 x 3 (narrower than the
    eq. (18) stencil, so every difference wraps).  The second call reads no
    stale partial of the first."""
    import torch
    stream = torch.cuda.current_stream()
    for nx, ny, seed in ((512, 512, 21), (5, 3, 22), (37, 23, 23)):
        m = P.Member(nx, ny, 0.61, 1.0, 1, 1, 3e-4, 2e-3)
        f = li.random_populations(nx, ny, seed=seed, rel_noise=0.03)
        got = _static_call(P, torch.from_numpy(f).cuda(), m, stream)
        want = orc.global_quantities(f, 0.61, orc.Force(1, 3e-4, 1, 2e-3))
        _compare(got, want, nx * ny)
        lat = P.Lattice([m], precision=64)
        lat.set_populations(0, f)
        _compare(got, lat.global_balance(0), nx * ny)
        lat.close()


def test_static_rejects_oversized_grid(P):
    import torch
    lib = P.load_library()
    m = P.Member(1024, 512, 0.6)
    cfg = m.c()
    out = np.zeros(P.NGLOBAL)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.lbm_global_balance_static(ctypes.c_void_p(dummy.data_ptr()), 1024, 512,
                                       ctypes.byref(cfg), out.ctypes.data_as(ctypes.c_void_p),
                                       None)
    assert rc == -1
    assert b"LBM_STATIC_MAX_CELLS" in lib.lbm_static_last_error()
