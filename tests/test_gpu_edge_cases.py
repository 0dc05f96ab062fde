"""Edge cases of the step and of the sub-volume balance through the C ABI:
a zero step count, rejected arguments (the handle stays usable and its
results unchanged), the extreme box sizes L = 1 (single cells) and L = N
(the whole periodic domain from every origin) against the FP64 oracle, and
the degenerate flow at rest whose balancing errors are 0/0 (eqs. 12, 13:
reported as 0)."""
import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu

TERM_TOL = 1e-10  # FP64 diagnostic, relative to each term field's maximum


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def _init(lat, nx, ny, seed):
    lat.init_fields(0, 1.0 + li.smooth_fields(nx, ny, seed, amp=0.01),
                    li.smooth_fields(nx, ny, seed + 1, amp=0.03),
                    li.smooth_fields(nx, ny, seed + 2, amp=0.03))


@pytest.mark.parametrize("prec", [32, 64])
def test_step_zero_is_a_noop_and_negative_is_rejected(P, prec):
    nx, ny = 32, 24
    lat = P.Lattice([P.Member(nx, ny, 0.57, 1.0, 1, 2, 2e-4, 1e-3)], precision=prec)
    _init(lat, nx, ny, 10)
    lat.step(3)
    f, t = lat.get_populations_host(0), lat.time
    lat.step(0)
    assert lat.time == t and np.array_equal(lat.get_populations_host(0), f)
    with pytest.raises(P.LBMError) as e:
        lat.step(-1)
    assert e.value.code == -1
    assert lat.time == t and np.array_equal(lat.get_populations_host(0), f)
    lat.close()


def test_balance_argument_errors_leave_the_handle_usable(P):
    n = 16
    lat = P.Lattice([P.Member(n, n, 0.6, 1.0, 1, 1, 2e-4, 0.0)], precision=64, diag_every=4)
    _init(lat, n, n, 20)
    lat.step(4)
    good = lat.subvolume_balance(0, [2, 5])
    o = np.array([[0, 0], [3, 7]], dtype=np.int32)
    bad = [
        dict(Ls=[]),                                       # no box size
        dict(Ls=list(range(1, 34))),                       # more than 32 sizes
        dict(Ls=[2], origins=np.array([[n, 0]])),          # x0 outside the grid
        dict(Ls=[2], origins=np.array([[0, -1]])),         # y0 outside the grid
        dict(Ls=[2, 3], origins=[o, np.zeros((0, 2))]),    # a size without boxes
    ]
    for kw in bad:
        with pytest.raises(P.LBMError) as e:
            lat.subvolume_balance(0, **kw)
        assert e.value.code == -1, kw
    # no such member: the C entry point itself rejects it
    Ls = np.array([2], dtype=np.int32)
    stats = np.empty((1, 15, 2))
    assert lat.lib.lbm_subvolume_balance(lat.h, 1, Ls.ctypes.data, 1, None, None,
                                         stats.ctypes.data, None) == -1
    assert lat.lib.lbm_subvolume_balance(lat.h, -1, Ls.ctypes.data, 1, None, None,
                                         stats.ctypes.data, None) == -1
    assert np.array_equal(lat.subvolume_balance(0, [2, 5]), good, equal_nan=True)
    lat.close()


def test_single_cell_and_whole_domain_boxes(P, orc):
    """L = 1: every box is one cell, so the per-box terms are the oracle's
    term fields cell by cell; L = N: every origin sees the whole periodic
    domain, so all boxes are equal (exact fixed-point sums: zero spread) and
    their mean is each term's global mean (forced flow, FP64)."""
    n, tau = 16, 0.56
    force = orc.Force(1, 3e-4, 1, 1e-3)
    lat = P.Lattice([P.Member(n, n, tau, 1.0, 1, 1, 3e-4, 1e-3)], precision=64)
    _init(lat, n, n, 30)
    lat.step(10)
    lat.record_snapshot()
    f10 = lat.get_populations_host(0)
    lat.step(1)
    lat.record_snapshot()
    f11 = lat.get_populations_host(0)
    lat.step(1)
    f12 = lat.get_populations_host(0)
    stats, pb = lat.subvolume_balance(0, [1, n], per_box=True)
    pb = pb.cpu().numpy().reshape(2, n * n, 15)
    T = orc.terms_from_populations(f12, f11, f10, tau, force)
    scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300  # RHS^{Omega,6} = 0 in 2D
    # L = 1, origin o = y * n + x: the cell (x, y)
    cells = T.reshape(13, -1).T
    assert np.max(np.abs(pb[0][:, 2:] - cells) / scale) < TERM_TOL
    # L = N: identical boxes, the global means
    assert np.all(pb[1][:, 2:] == pb[1][:1, 2:])
    assert np.all(stats[1, 2:, 1] <= TERM_TOL * scale)  # spread of equal boxes
    np.testing.assert_allclose(stats[1, 2:, 0], T.reshape(13, -1).mean(axis=1), rtol=0,
                               atol=TERM_TOL * np.max(scale))
    np.testing.assert_allclose(stats[0, 2:, 0], stats[1, 2:, 0], rtol=0,
                               atol=TERM_TOL * np.max(scale))
    lat.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_flow_at_rest_balancing_errors_are_zero(P, prec):
    """Uniform density at rest: every term vanishes, so the balancing errors
    of eqs. (12), (13) are 0/0, reported as 0 (not NaN) for every box."""
    n = 16
    lat = P.Lattice([P.Member(n, n, 0.6)], precision=prec, diag_every=2)
    lat.init_fields(0, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    lat.step(4)
    stats, pb = lat.subvolume_balance(0, [1, 4, n], per_box=True)
    assert np.all(stats == 0.0)
    assert np.all(pb.cpu().numpy() == 0.0)
    lat.close()
