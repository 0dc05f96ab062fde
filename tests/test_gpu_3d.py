"""GPU parity of the three-dimensional extension (D3Q19 and D3Q27 BGK with EDM forcing;
the general-index balance terms with vortex stretching over L^3 boxes)
against the FP64 oracle, through the C ABI of include/lbm3d.h: trajectories
(FP64 within 1e-12, FP32 within 2e-6 on every population), state round
trips, and the box terms and statistics on the GPU's exported states."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TERM_TOL = 1e-10


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def rel_err(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


def _smooth3(shape, seed, amp):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(2 * np.pi * np.arange(nz) / nz, 2 * np.pi * np.arange(ny) / ny,
                          2 * np.pi * np.arange(nx) / nx, indexing="ij")
    out = np.zeros(shape)
    for _ in range(4):
        k = rng.integers(-2, 3, size=3)
        out += rng.normal() * np.cos(k[0] * X + k[1] * Y + k[2] * Z + rng.uniform(0, 2 * np.pi))
    return amp * out / np.max(np.abs(out))


def _fields(shape, seed):
    return (1.0 + _smooth3(shape, seed, 0.01), _smooth3(shape, seed + 1, 0.04),
            _smooth3(shape, seed + 2, 0.04), _smooth3(shape, seed + 3, 0.04))


SPEC = [(12, 10, 8, 0.57, 1, 1, 3e-4, 2e-3), (16, 16, 16, 0.52, 0, 0, 0.0, 0.0),
        (5, 7, 3, 0.8, 1, 1, 1e-4, 0.0)]


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-6)])
def test_3d_trajectories(P, orc, prec, tol, q):
    lat = P.Lattice3D([P.Member3(nx, ny, nz, tau, 1.0, k, kf, F0, a)
                       for (nx, ny, nz, tau, k, kf, F0, a) in SPEC], precision=prec, lattice=q)
    init = []
    for i, (nx, ny, nz, *_r) in enumerate(SPEC):
        fl = _fields((nz, ny, nx), 10 * i)
        lat.init_fields(i, *fl)
        init.append(orc.init3(*fl, q=q))
    done = 0
    ref = list(init)
    for steps in (1, 5, 24, 100):  # up to the 100-step population parity horizon
        lat.step(steps - done)
        for i, (nx, ny, nz, tau, k, kf, F0, a) in enumerate(SPEC):
            ref[i] = orc.run3(ref[i], steps - done, tau, k, F0, kf, a)
            err = rel_err(lat.get_populations_host(i), ref[i])
            assert err < tol, (prec, steps, i, err)
        done = steps


SPEC_VEC = [(12, 10, 8, 0.57, 1, 1, 3e-4, 2e-3), (132, 6, 4, 0.53, 1, 2, 2e-4, 0.0),
            (64, 5, 3, 0.6, 0, 0, 0.0, 0.0)]


@pytest.mark.parametrize("q", [19, 27])
@pytest.mark.parametrize("cpl", [4, 2])
def test_3d_cells_per_lane(P, orc, q, cpl):
    """The vectorised FP32 kernel with 4 and with 2 cells per lane (128- and
    64-cell row segments: widths 12, 64 and 132 leave partial segments and a
    4-cell remainder) against the oracle at the FP32 bar over 100 steps."""
    lat = P.Lattice3D([P.Member3(nx, ny, nz, tau, 1.0, k, kf, F0, a)
                       for (nx, ny, nz, tau, k, kf, F0, a) in SPEC_VEC], precision=32, lattice=q)
    lat.set_cells_per_lane(cpl)
    assert lat.tuning()["cells_per_lane"] == cpl
    with pytest.raises(RuntimeError):
        lat.set_cells_per_lane(3)
    assert lat.tuning()["cells_per_lane"] == cpl
    ref = []
    for i, (nx, ny, nz, *_r) in enumerate(SPEC_VEC):
        fl = _fields((nz, ny, nx), 40 + 10 * i)
        lat.init_fields(i, *fl)
        ref.append(orc.init3(*fl, q=q))
    done = 0
    for steps in (1, 5, 100):
        lat.step(steps - done)
        for i, (nx, ny, nz, tau, k, kf, F0, a) in enumerate(SPEC_VEC):
            ref[i] = orc.run3(ref[i], steps - done, tau, k, F0, kf, a)
            err = rel_err(lat.get_populations_host(i), ref[i])
            assert err < 2e-6, (q, cpl, steps, i, err)
        done = steps


@pytest.mark.parametrize("q", [19, 27])
def test_3d_state_roundtrip(P, orc, q):
    shape = (6, 5, 7)
    f = orc.init3(*_fields(shape, 3), q=q) * (
        1 + 0.01 * np.random.default_rng(1).normal(size=(q,) + shape))
    lat = P.Lattice3D([P.Member3(7, 5, 6, 0.6)], precision=64, lattice=q)
    lat.set_populations(0, f)
    assert np.array_equal(lat.get_populations_host(0), f)
    lat.step(3)
    assert rel_err(lat.get_populations_host(0), orc.run3(f, 3, 0.6)) < 1e-12


@pytest.mark.parametrize("prec,q", [(64, 19), (32, 19), (64, 27), (32, 27)])
def test_3d_balance_terms(P, orc, prec, q):
    """All origins and origin lists at several L (one beyond the grid: NaN);
    per-box terms within 1e-10 of each field's magnitude of the oracle's on
    the same exported states; vortex stretching is present."""
    nx, ny, nz, tau, F0, kf, a = 12, 10, 8, 0.57, 3e-4, 1, 2e-3
    lat = P.Lattice3D([P.Member3(nx, ny, nz, tau, 1.0, 1, kf, F0, a)], precision=prec,
                      diag_every=10, lattice=q)
    lat.init_fields(0, *_fields((nz, ny, nx), 40))
    lat.step(8)
    f8 = lat.get_populations_host(0)
    lat.step(1)
    f9 = lat.get_populations_host(0)
    lat.step(1)
    f10 = lat.get_populations_host(0)
    T = orc.terms3_from_populations(f10, f9, f8, tau, 1, F0, kf, a)
    scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
    assert scale[12] > 1e-6 * scale[8]  # RHS^{O,6} does not vanish in 3D
    Ls = [1, 3, 8]
    stats, pb = lat.subvolume_balance(0, Ls, per_box=True)
    pb = pb.cpu().numpy().reshape(len(Ls), -1, 15)
    want, want_pb = orc.balance_stats3(T, Ls, per_box=True)
    for iL in range(len(Ls)):
        d = np.abs(pb[iL][:, 2:] - want_pb[iL][:, 2:]) / scale[None, :]
        assert np.max(d) < TERM_TOL, (Ls[iL], np.max(d))
        np.testing.assert_allclose(stats[iL, 2:, 0], want[iL, 2:, 0], rtol=0,
                                   atol=TERM_TOL * np.max(scale))
    rng = np.random.default_rng(2)
    origins = [np.stack([rng.integers(0, nx, 50), rng.integers(0, ny, 50), rng.integers(0, nz, 50)], 1)
               for _ in range(3)]
    Ls2 = [2, 5, 9]
    st2 = lat.subvolume_balance(0, Ls2, origins=origins)
    assert np.all(np.isnan(st2[2]))
    for iL in range(2):
        w = orc.balance_stats3(T, [Ls2[iL]], origins=origins[iL])
        np.testing.assert_allclose(st2[iL, 2:, 0], w[0, 2:, 0], rtol=0, atol=TERM_TOL * np.max(scale))
        np.testing.assert_allclose(st2[iL, :2, 0], w[0, :2, 0], rtol=1e-6, atol=1e-8)


# FP32 balance arithmetic: the level differences are formed in FP64 from the
# FP64 snapshots and rounded once; the remaining error is the FP32 rounding
# amplified by the nested eq. (18) differences (three for RHS^{O,4} and
# RHS^{O,5}), as in two dimensions: bar 1e-4 of each field's magnitude.
FP32_TERM_TOL = 1e-4


@pytest.mark.parametrize("prec,q", [(32, 19), (32, 27), (64, 19)])
def test_3d_balance_terms_fp32_arithmetic(P, orc, prec, q):
    """diag_precision 32: per-box terms within 1e-4 of each field's
    magnitude of the oracle's on the same exported states (all origins and
    an origin list), balancing-error statistics within 1e-3 relative; vortex
    stretching present."""
    nx, ny, nz, tau, F0, kf, a = 16, 12, 10, 0.57, 3e-4, 1, 2e-3
    lat = P.Lattice3D([P.Member3(nx, ny, nz, tau, 1.0, 1, kf, F0, a)], precision=prec,
                      diag_every=10, lattice=q, diag_precision=32)
    lat.init_fields(0, *_fields((nz, ny, nx), 60))
    lat.step(8)
    f8 = lat.get_populations_host(0)
    lat.step(1)
    f9 = lat.get_populations_host(0)
    lat.step(1)
    f10 = lat.get_populations_host(0)
    T = orc.terms3_from_populations(f10, f9, f8, tau, 1, F0, kf, a)
    scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
    assert scale[12] > 1e-6 * scale[8]
    Ls = [1, 3, 8]
    stats, pb = lat.subvolume_balance(0, Ls, per_box=True)
    pb = pb.cpu().numpy().reshape(len(Ls), -1, 15)
    want, want_pb = orc.balance_stats3(T, Ls, per_box=True)
    for iL in range(len(Ls)):
        d = np.abs(pb[iL][:, 2:] - want_pb[iL][:, 2:]) / scale[None, :]
        assert np.max(d) < FP32_TERM_TOL, (Ls[iL], np.max(d))
        np.testing.assert_allclose(stats[iL, 2:, 0], want[iL, 2:, 0], rtol=0,
                                   atol=FP32_TERM_TOL * np.max(scale))
    rng = np.random.default_rng(3)
    origins = [np.stack([rng.integers(0, nx, 60), rng.integers(0, ny, 60),
                         rng.integers(0, nz, 60)], 1) for _ in range(2)]
    st2 = lat.subvolume_balance(0, [4, 9], origins=origins)
    for iL, L in enumerate([4, 9]):
        w = orc.balance_stats3(T, [L], origins=origins[iL])
        np.testing.assert_allclose(st2[iL, 2:, 0], w[0, 2:, 0], rtol=0,
                                   atol=FP32_TERM_TOL * np.max(scale))
        np.testing.assert_allclose(st2[iL, :2, 0], w[0, :2, 0], rtol=1e-3)


def test_3d_history_required(P):
    lat = P.Lattice3D([P.Member3(8, 8, 8, 0.6)], precision=64)
    lat.init_fields(0, np.ones((8, 8, 8)), *(np.zeros((8, 8, 8)) for _ in range(3)))
    lat.step(4)
    with pytest.raises(P.LBMError) as e:
        lat.subvolume_balance(0, [2])
    assert e.value.code == -4


@pytest.mark.parametrize("q", [19, 27])
def test_3d_edge_cases(P, orc, q):
    """Zero steps are a no-op and a negative count is rejected; rejected
    balance arguments leave the handle usable; L = N boxes (the whole
    periodic cube from every origin) are all equal, with the global means of
    the oracle's terms; a flow at rest has zero terms and zero balancing
    errors (eqs. 12, 13 at 0/0)."""
    n, tau, F0, kf, a = 8, 0.58, 3e-4, 1, 2e-3
    lat = P.Lattice3D([P.Member3(n, n, n, tau, 1.0, 1, kf, F0, a)], precision=64, diag_every=4,
                      lattice=q)
    lat.init_fields(0, *_fields((n, n, n), 70))
    lat.step(2)
    f2 = lat.get_populations_host(0)
    lat.step(0)
    assert lat.time == 2 and np.array_equal(lat.get_populations_host(0), f2)
    with pytest.raises(P.LBMError) as e:
        lat.step(-1)
    assert e.value.code == -1 and lat.time == 2
    lat.step(1)
    f3 = lat.get_populations_host(0)
    lat.step(1)
    f4 = lat.get_populations_host(0)
    for kw in (dict(Ls=[]), dict(Ls=[2], origins=[np.array([[n, 0, 0]])]),
               dict(Ls=[2], origins=[np.array([[0, 0, -1]])])):
        with pytest.raises(P.LBMError) as e:
            lat.subvolume_balance(0, **kw)
        assert e.value.code == -1, kw
    stats, pb = lat.subvolume_balance(0, [n], per_box=True)
    pb = pb.cpu().numpy()
    T = orc.terms3_from_populations(f4, f3, f2, tau, 1, F0, kf, a)
    scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
    assert pb.shape[0] == n ** 3 and np.all(pb[:, 2:] == pb[:1, 2:])
    np.testing.assert_allclose(stats[0, 2:, 0], T.reshape(13, -1).mean(axis=1), rtol=0,
                               atol=TERM_TOL * np.max(scale))
    lat.close()
    rest = P.Lattice3D([P.Member3(n, n, n, 0.6)], precision=64, diag_every=2, lattice=q)
    rest.init_fields(0, np.ones((n, n, n)), *(np.zeros((n, n, n)) for _ in range(3)))
    rest.step(4)
    st, pbr = rest.subvolume_balance(0, [1, 4, n], per_box=True)
    assert np.all(st == 0.0) and np.all(pbr.cpu().numpy() == 0.0)
    rest.close()
