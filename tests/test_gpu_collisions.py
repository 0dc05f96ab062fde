"""GPU parity of the variable-viscosity collisions (Sec. 1: the Smagorinsky
eddy viscosity and the turbulent viscosity of eq. (7), each a local
relaxation time from the non-equilibrium stress, and the entropic LBM with
its per-cell entropy-condition root) against the FP64 oracle,
through the C ABI: trajectories (FP64 within 1e-12, FP32 within 2e-6 on
every population) in mixed ensembles on both kernels and both storages, the
whole-grid budget with the local viscosity, and the balance terms whose
viscous terms use the local viscosity of each cell at time n."""
import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-6
TERM_TOL = 1e-10
CS = 0.15  # Smagorinsky constant of the tests (dx = 1)


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def rel_err(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


def _fields(nx, ny, seed, amp=0.05):
    return (1.0 + li.smooth_fields(nx, ny, seed + 2, amp=0.02),
            li.smooth_fields(nx, ny, seed, amp=amp), li.smooth_fields(nx, ny, seed + 1, amp=amp))


# (nx, ny, tau, force kind, F0, kf, alpha, collision): vector and general
# kernels, every force kind (the entropic collision with each of them)
SPEC = [(64, 48, 0.51, 0, 0.0, 0, 0.0, 1), (37, 23, 0.53, 1, 2e-4, 2, 1e-3, 1),
        (48, 40, 0.52, 2, 2e-5, 0, 0.0, 2), (32, 32, 0.55, 1, 2e-4, 2, 0.0, 2),
        (40, 40, 0.56, 0, 0.0, 0, 0.0, 0), (48, 40, 0.505, 0, 0.0, 0, 0.0, 3),
        (37, 23, 0.51, 1, 2e-4, 2, 1e-3, 3), (48, 40, 0.51, 2, 2e-5, 0, 0.0, 3),
        (37, 23, 0.52, 2, 2e-5, 0, 0.0, 3)]


def _member(P, spec):
    nx, ny, tau, k, F0, kf, a, coll = spec
    return P.Member(nx, ny, tau, 1.0, k, kf, F0, a, 0.6 if k == 2 else 0.0,
                    2e-2 if k == 2 else 0.0, coll, CS if coll == 1 else 0.0)


def _model(orc, spec):
    nx, ny, tau, k, F0, kf, a, coll = spec
    return orc.Force(k, F0, kf, a, phase=0.6 if k == 2 else 0.0, FR0=2e-2 if k == 2 else 0.0,
                     collision=coll, Cs=CS if coll == 1 else 0.0)


CHECKPOINTS = (1, 8, 31, 100)  # up to the 100-step population parity horizon


@pytest.fixture(scope="module")
def oracle_trajectories(orc):
    """Oracle states of every SPEC member at the checkpoint steps, from the
    oracle's own equilibrium of the initial fields."""
    out = []
    for i, sp in enumerate(SPEC):
        f, done, states = orc.init(*_fields(sp[0], sp[1], 7 * i + 1)), 0, {}
        for steps in CHECKPOINTS:
            f = orc.run(f, steps - done, sp[2], _model(orc, sp))
            done = steps
            states[steps] = f
        out.append(states)
    return out


@pytest.mark.parametrize("prec,tol", [(64, FP64_TOL), (32, FP32_TOL)])
@pytest.mark.parametrize("storage", [1, 2])
def test_collision_trajectories(P, oracle_trajectories, prec, tol, storage):
    lat = P.Lattice([_member(P, sp) for sp in SPEC], precision=prec, storage=storage,
                    graph_steps=6)
    for i, sp in enumerate(SPEC):
        lat.init_fields(i, *_fields(sp[0], sp[1], 7 * i + 1))
    done = 0
    for steps in CHECKPOINTS:
        lat.step(steps - done)
        done = steps
        for i, sp in enumerate(SPEC):
            err = rel_err(lat.get_populations_host(i), oracle_trajectories[i][steps])
            assert err < tol, (prec, storage, steps, i, err)


@pytest.mark.parametrize("nx", [32, 33])
@pytest.mark.parametrize("prec,tol", [(64, FP64_TOL), (32, FP32_TOL)])
def test_elbm_far_from_equilibrium(P, orc, prec, tol, nx):
    """ELBM steps from a state with half its cells departing from the
    entropic equilibrium by up to 12% (relative departures y above 0.02: the
    FP32 root takes Newton's iteration) and half near it (y below 0.01: the
    root's series alone), one and three steps against the oracle, without
    and with the force and drag; nx = 32 runs FP32 on the vectorised kernel,
    nx = 33 on the general one."""
    ny, tau = 24, 0.52
    rng = np.random.default_rng(5)
    f0 = orc.init(*_fields(nx, ny, 11))
    hit = rng.uniform(size=(1, ny, nx)) < 0.5
    f0 = f0 * (1.0 + 0.12 * rng.uniform(-1.0, 1.0, size=f0.shape) * hit)
    cx, cy, _ = orc.lattice()
    ymax = np.empty((ny, nx))
    for j in range(ny):
        for i in range(nx):
            f = f0[:, j, i]
            rho = f.sum()
            d = orc.feq_entropic(rho, (cx * f).sum() / rho, (cy * f).sum() / rho) - f
            ymax[j, i] = np.abs(d / f).max()
    assert (ymax > 0.03).mean() > 0.3 and (ymax < 0.01).mean() > 0.3
    for kind, F0, alpha in ((0, 0.0, 0.0), (1, 2e-4, 1e-3)):
        lat = P.Lattice([P.Member(nx, ny, tau, 1.0, kind, 2, F0, alpha, 0.0, 0.0, 3, 0.0)],
                        precision=prec)
        lat.set_populations(0, f0)
        model = orc.Force(kind, F0, 2, alpha, collision=3)
        done = 0
        for steps in (1, 3):
            lat.step(steps - done)
            done = steps
            err = rel_err(lat.get_populations_host(0), orc.run(f0, steps, tau, model))
            assert err < tol, (prec, kind, steps, err)


def test_collision_models_change_the_flow(P, orc):
    """Both models move the state by far more than the parity bar relative to
    BGK (eq. (7) through the compressible part of the strain)."""
    nx, ny, tau = 48, 40, 0.51
    f = orc.init(*_fields(nx, ny, 3))
    bgk = orc.run(f, 20, tau)
    for coll, cs in ((1, CS), (2, 0.0), (3, 0.0)):
        other = orc.run(f, 20, tau, orc.Force(0, collision=coll, Cs=cs))
        assert rel_err(other, bgk) > 50 * FP32_TOL, coll


@pytest.mark.parametrize("coll", [1, 2, 3])
def test_collision_budget_and_balance_terms(P, orc, coll):
    nx, ny, tau = 64, 48, 0.52
    model = orc.Force(1, 2e-4, 2, 1e-3, collision=coll, Cs=CS if coll == 1 else 0.0)
    lat = P.Lattice([P.Member(nx, ny, tau, 1.0, 1, 2, 2e-4, 1e-3, 0.0, 0.0, coll,
                              CS if coll == 1 else 0.0)], precision=64, diag_every=24)
    lat.init_fields(0, *_fields(nx, ny, 11))
    lat.step(22)
    f22 = lat.get_populations_host(0)
    lat.step(1)
    f23 = lat.get_populations_host(0)
    lat.step(1)
    f24 = lat.get_populations_host(0)
    g = lat.global_balance(0)
    gw = orc.global_quantities(f24, tau, model)
    np.testing.assert_allclose(g[[0, 3, 4, 5, 6]], gw[[0, 3, 4, 5, 6]], rtol=1e-12)
    Ls = [1, 4, 16, 48]
    stats, pb = lat.subvolume_balance(0, Ls, per_box=True)
    pb = pb.cpu().numpy().reshape(len(Ls), -1, 15)
    T = orc.terms_from_populations(f24, f23, f22, tau, model)
    want, want_pb = orc.balance_stats(T, Ls, per_box=True)
    scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
    for iL in range(len(Ls)):
        d = np.abs(pb[iL][:, 2:] - want_pb[iL][:, 2:]) / scale[None, :]
        assert np.max(d) < TERM_TOL, (Ls[iL], np.max(d))
    # the local viscosity matters: the constant-viscosity terms differ
    T_bgk = orc.terms_from_populations(f24, f23, f22, tau, orc.Force(1, 2e-4, 2, 1e-3))
    assert np.max(np.abs(T_bgk[4] - T[4])) > 1e4 * TERM_TOL * scale[4]


@pytest.mark.parametrize("coll", [1, 3])
def test_fp32_collision_diagnostic(P, orc, coll):
    """FP32 storage and diagnostic with the Smagorinsky model and ELBM: box
    terms within the FP32 bar of the oracle on the exported states."""
    nx, ny, tau = 64, 64, 0.51
    cs = CS if coll == 1 else 0.0
    model = orc.Force(0, collision=coll, Cs=cs)
    lat = P.Lattice([P.Member(nx, ny, tau, 1.0, 0, 0, 0.0, 0.0, 0.0, 0.0, coll, cs)],
                    precision=32, diag_every=16)
    lat.init_fields(0, *_fields(nx, ny, 21))
    lat.step(14)
    f14 = lat.get_populations_host(0)
    lat.step(1)
    f15 = lat.get_populations_host(0)
    lat.step(1)
    f16 = lat.get_populations_host(0)
    Ls = [2, 8, 32]
    stats, pb = lat.subvolume_balance(0, Ls, per_box=True)
    pb = pb.cpu().numpy().reshape(len(Ls), -1, 15)
    T = orc.terms_from_populations(f16, f15, f14, tau, model)
    _, want_pb = orc.balance_stats(T, Ls, per_box=True)
    scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
    for iL in range(len(Ls)):
        d = np.abs(pb[iL][:, 2:] - want_pb[iL][:, 2:]) / scale[None, :]
        assert np.max(d) < 1e-4, (Ls[iL], np.max(d))


def test_adjoint_rejects_variable_viscosity(P):
    import torch
    n = 16
    lat = P.Lattice([P.Member(n, n, 0.6, 1.0, 0, 0, 0.0, 0.0, 0.0, 0.0, 1, CS)], precision=64)
    lat.init_fields(0, *_fields(n, n, 1))
    f = lat.get_populations(0)
    lam = torch.zeros_like(f)
    out = torch.empty_like(f)
    acc = torch.zeros(2, dtype=torch.float64, device=f.device)
    with pytest.raises(P.LBMError) as e:
        lat.adjoint_step(0, f, lam, out, 1.0, (0, 0), 4, acc[0:1], acc[1:2])
    assert e.value.code == -1
