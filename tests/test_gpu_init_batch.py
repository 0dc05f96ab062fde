"""lbm_init_fields_batch against lbm_init_fields member by member: the same
populations bit for bit from host fields (chunked through the staging
scratch when the members do not fit it at once) and from device fields,
for a subset of members too, and the argument checks."""
import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def _fields(n, nx, ny, seed):
    r = np.stack([1.0 + li.smooth_fields(nx, ny, seed + 3 * i, amp=0.01) for i in range(n)])
    u = np.stack([li.smooth_fields(nx, ny, seed + 3 * i + 1, amp=0.03) for i in range(n)])
    v = np.stack([li.smooth_fields(nx, ny, seed + 3 * i + 2, amp=0.03) for i in range(n)])
    return r, u, v


@pytest.mark.parametrize("prec,storage", [(32, 1), (32, 2), (64, 2)])
def test_batch_equals_per_member(P, prec, storage):
    import torch
    n, nx, ny = 24, 32, 32  # with diag_batch = 1 the staging holds about 20 members
    members = [P.Member(nx, ny, 0.55 + 0.01 * (i % 3)) for i in range(n)]
    r, u, v = _fields(n, nx, ny, 500)
    a = P.Lattice(members, precision=prec, storage=storage, diag_batch=1)
    b = P.Lattice(members, precision=prec, storage=storage, diag_batch=1)
    c = P.Lattice(members, precision=prec, storage=storage, diag_batch=1)
    for m in range(n):
        a.init_fields(m, r[m], u[m], v[m])
    b.init_fields_batch(list(range(n)), r, u, v)
    c.init_fields_batch(list(range(n)), *(torch.from_numpy(x).cuda() for x in (r, u, v)))
    for m in range(n):
        fa = a.get_populations_host(m)
        assert np.array_equal(fa, b.get_populations_host(m)), m
        assert np.array_equal(fa, c.get_populations_host(m)), m
    for lat in (a, b, c):
        lat.step(5)
    for m in (0, 7, n - 1):
        assert np.array_equal(a.get_populations_host(m), b.get_populations_host(m))
    # a subset in any order, the others untouched (double buffer, or AA at an
    # even step; at an odd step AA storage needs every member listed)
    sub = [5, 2, 17]
    r2, u2, v2 = _fields(len(sub), nx, ny, 900)
    if storage == 1:
        with pytest.raises(P.LBMError):
            b.init_fields_batch(sub, r2, u2, v2)  # time 5: odd
    a.step(1)
    b.step(1)
    keep = b.get_populations_host(3)
    for i, m in enumerate(sub):
        a.init_fields(m, r2[i], u2[i], v2[i])
    b.init_fields_batch(sub, r2, u2, v2)
    for m in sub + [3]:
        assert np.array_equal(a.get_populations_host(m), b.get_populations_host(m))
    assert np.array_equal(b.get_populations_host(3), keep)


def test_batch_argument_checks(P):
    lat = P.Lattice([P.Member(32, 32, 0.6), P.Member(32, 32, 0.6), P.Member(16, 32, 0.6)])
    r, u, v = _fields(2, 32, 32, 1)
    with pytest.raises(P.LBMError):
        lat.init_fields_batch([0, 0], r, u, v)  # listed twice
    with pytest.raises(P.LBMError):
        lat.init_fields_batch([0, 2], r, u, v)  # unequal grids
    with pytest.raises(P.LBMError):
        lat.init_fields_batch([0, 3], r, u, v)  # out of range
    lat.init_fields_batch([1, 0], r, u, v)
    assert lat.time == 0


def test_device_init_does_not_disturb_queued_diagnostic(P):
    """A device-field (re)initialisation queued right after an asynchronous
    diagnostic does not wait for it and does not change its statistics: the
    diagnostic works on the snapshot ring, the initialisation on the
    populations."""
    import torch
    n, M, D = 64, 4, 20
    members = [P.Member(n, n, 0.55)] * M
    r, u, v = _fields(M, n, n, 40)
    dev = [torch.from_numpy(x).cuda() for x in (r, u, v)]
    Ls = [2, 4, 8, 16]
    a = P.Lattice(members, precision=32, diag_every=D)
    b = P.Lattice(members, precision=32, diag_every=D)
    for lat in (a, b):
        lat.init_fields_batch(list(range(M)), *dev)
        lat.step(D)
    want = b.subvolume_balance_batch(list(range(M)), Ls)
    out = a.subvolume_balance_async(list(range(M)), Ls)
    r2, u2, v2 = _fields(M, n, n, 41)
    a.init_fields_batch(list(range(M)), *(torch.from_numpy(x).cuda() for x in (r2, u2, v2)))
    a.step(3)
    a.diag_synchronize()
    assert np.array_equal(out.cpu().numpy(), want, equal_nan=True)
    c = P.Lattice(members, precision=32)
    c.init_fields_batch(list(range(M)), r2, u2, v2)
    c.step(3)
    for m in range(M):
        assert np.array_equal(a.get_populations_host(m), c.get_populations_host(m))
