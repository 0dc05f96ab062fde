"""GPU checks of the hand-written adjoint (no counterpart in the paper):
the transposed step against finite differences of the FP64 GPU forward
(dot-product test), and the checkpointed gradients of the box-averaged
dissipation objective against central finite differences of the FP64
oracle (bar: 1e-6 relative)."""
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


def test_adjoint_step_dot_product(P):
    """<lam, dS(f)[d]> = <S^T lam, d> for one step, with dS[d] by central
    differences of the FP64 GPU step (no objective term)."""
    import torch
    nx, ny, tau, F0, kf, alpha = 24, 20, 0.57, 2e-4, 2, 3e-3
    lat = P.Lattice([P.Member(nx, ny, tau, 1.0, 1, kf, F0, alpha)], precision=64)
    f = torch.from_numpy(li.random_populations(nx, ny, seed=1)).cuda()
    rng = np.random.default_rng(2)
    d = torch.from_numpy(rng.standard_normal((9, ny, nx))).cuda()
    lam = torch.from_numpy(rng.standard_normal((9, ny, nx))).cuda()
    eps = 1e-6

    def S(x):
        lat.set_populations(0, x)
        lat.step(1)
        return lat.get_populations(0).clone()

    jv = (S(f + eps * d) - S(f - eps * d)) / (2 * eps)
    out = torch.empty_like(lam)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dF = torch.zeros(1, dtype=torch.float64, device="cuda")
    lat.adjoint_step(0, f, lam, out, 0.0, (0, 0), 1, dt, dF)
    lhs = float((lam * jv).sum())
    rhs = float((out * d).sum())
    assert abs(lhs - rhs) < 1e-7 * abs(rhs)

    # parameter directions: tau and F0
    def S_param(t, a):
        l2 = P.Lattice([P.Member(nx, ny, t, 1.0, 1, kf, a, alpha)], precision=64)
        l2.set_populations(0, f)
        l2.step(1)
        return l2.get_populations(0).clone()

    h = 1e-6
    dS_dtau = (S_param(tau + h, F0) - S_param(tau - h, F0)) / (2 * h)
    dS_dF0 = (S_param(tau, F0 * (1 + 1e-3)) - S_param(tau, F0 * (1 - 1e-3))) / (2e-3 * F0)
    assert abs(float((lam * dS_dtau).sum()) - float(dt)) < 1e-6 * abs(float(dt))
    assert abs(float((lam * dS_dF0).sum()) - float(dF)) < 1e-6 * abs(float(dF))


@pytest.mark.parametrize("nstates,weighted,box,L", [(7, (2, 3, 5), (35, 24), 8), (6, (), (35, 24), 8),
                                                   (1, (0,), (35, 24), 8),
                                                   (5, (1, 3), (30, 20), 24)])
def test_adjoint_sweep_matches_single_steps(P, nstates, weighted, box, L):
    """lbm_adjoint_sweep over a recorded interval (one gradient reduction per
    call, force-direction tables built once) against nstates single
    lbm_adjoint_step calls, last level first: the adjoint fields bit for
    bit, dJ/dtau and dJ/dF0 to the rounding of their FP64 sums (1e-13);
    objective weights on some levels, on none, and a one-level sweep with a
    zero incoming adjoint."""
    import torch
    nx, ny, tau, F0, kf, alpha = 40, 28, 0.56, 2e-4, 2, 1e-3
    # boxes wrapping around both edges; L = 24: a region of 32 x 28 cells
    lat = P.Lattice([P.Member(nx, ny, tau, 1.0, 1, kf, F0, alpha)], precision=64)
    lat.set_populations(0, torch.from_numpy(li.random_populations(nx, ny, seed=4)).cuda())
    states = torch.empty((nstates, 9, ny, nx), dtype=torch.float64, device="cuda")
    lat.record_trajectory(0, states)
    rng = np.random.default_rng(5)
    lam0 = None if nstates == 1 else torch.from_numpy(rng.standard_normal((9, ny, nx))).cuda()
    w = np.zeros(nstates)
    for k in weighted:
        w[k] = 0.1 * (k + 1)
    acc = torch.zeros(4, dtype=torch.float64, device="cuda")
    out, tmp = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda"), \
        torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    lat.adjoint_sweep(0, states, lam0, out, tmp, w, box, L, acc[0:1], acc[1:2])
    lam = lam0
    for k in range(nstates - 1, -1, -1):
        nxt = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
        lat.adjoint_step(0, states[k], lam, nxt, float(w[k]), box, L, acc[2:3], acc[3:4])
        lam = nxt
    assert torch.equal(out, lam)
    a = acc.cpu().numpy()
    assert abs(a[0] - a[2]) <= 1e-13 * abs(a[2]), (a[0], a[2])
    assert abs(a[1] - a[3]) <= 1e-13 * abs(a[3]), (a[1], a[3])
    with pytest.raises(RuntimeError):  # weights must be finite
        lat.adjoint_sweep(0, states, lam0, out, tmp, np.full(nstates, np.nan), box, L,
                          acc[0:1], acc[1:2])
    with pytest.raises(RuntimeError):  # box outside the grid with a weighted level
        lat.adjoint_sweep(0, states, lam0, out, tmp, np.ones(nstates), (nx, 0), L,
                          acc[0:1], acc[1:2])


@pytest.mark.parametrize("prec,grids", [(64, [(37, 23)]), (32, [(37, 23)]), (32, [(40, 24)]),
                                         (64, [(37, 23), (16, 12)])])
def test_record_trajectory_matches_steps(P, prec, grids):
    """lbm_record_trajectory against single steps and exports (lbm_step(1) +
    lbm_get_populations), bit for bit, and the handle's time afterwards: one
    member on the general kernel (each step writes the state it starts from,
    FP64 and FP32), one on the FP32 vector kernel and two members (step and
    export per level)."""
    import torch
    members = [P.Member(nx, ny, 0.57, 1.0, 1, 1, 2e-4, 1e-3) for (nx, ny) in grids]
    a = P.Lattice(members, precision=prec)
    b = P.Lattice(members, precision=prec)
    for i, (nx, ny) in enumerate(grids):
        f0 = torch.from_numpy(li.random_populations(nx, ny, seed=20 + i)).cuda()
        a.set_populations(i, f0)
        b.set_populations(i, f0)
    a.step(3)
    b.step(3)
    K = 9
    nx, ny = grids[0]
    states = torch.empty((K, 9, ny, nx), dtype=torch.float64, device="cuda")
    a.record_trajectory(0, states)
    for k in range(K):
        if k:
            b.step(1)
        assert torch.equal(states[k], b.get_populations(0)), k
    assert a.time == b.time == 3 + K - 1
    a.step(2)
    b.step(2)
    for i in range(len(grids)):
        assert torch.equal(a.get_populations(i), b.get_populations(i))


def _small_spec(precision=64):
    from paper_1809_06735_gb300.adjoint import ObjectiveSpec
    return ObjectiveSpec(nx=32, ny=32, kf=2, alpha=1e-3, n0=20, n1=44, box=(5, 3), L=8,
                         precision=precision, checkpoint_every=10)


@pytest.mark.parametrize("n,box,L,precision,tol", [
    (32, (5, 3), 8, 64, 1e-12),       # 4 x 4 tiles: 2 x 2 CTAs
    (32, (29, 30), 8, 64, 1e-12),     # the same, box wrapping around both edges
    (48, (3, 40), 30, 64, 1e-12),     # ragged last tiles (30 = 7 x 4 + 2)
    (48, (10, 2), 45, 64, 1e-12),     # the stencil reach wraps onto the box itself
    (128, (100, 7), 101, 64, 1e-12),  # 8 x 8 tiles (13 x 13 CTAs), ragged, wrapping
    (200, (150, 190), 197, 64, 1e-12),  # 16 x 16 tiles (13 x 13 CTAs), ragged, wrapping
    (520, (7, 500), 515, 64, 1e-12),  # 33 x 33 tiles on 1024 CTAs (a CTA does two)
    (6, (4, 5), 6, 64, 1e-12),        # a grid smaller than one widened tile: halos wrap twice
    (32, (5, 3), 8, 32, 1e-5),        # FP32 populations
    (200, (150, 190), 197, 32, 1e-5)])  # FP32, 16 x 16 tiles
def test_objective_forward_matches_oracle(P, orc, n, box, L, precision, tol):
    """J over n in [20, 44] against the oracle's objective: every tile size
    of the one-launch objective (4, 8, 16), ragged last tiles, boxes across
    the periodic edges, a stencil reach that wraps onto the box, more tiles
    than CTAs.  FP32 populations: the storage rounding of a 44-step
    trajectory."""
    import dataclasses
    import torch
    from paper_1809_06735_gb300.adjoint import forward_objective
    spec = dataclasses.replace(_small_spec(precision), nx=n, ny=n, box=box, L=L)
    tau, F0 = 0.6, li.kolmogorov_F0(n, 0.6, 2, 1e-3, 0.02)
    r, u, v = li.random_phase(n, seed=4, u_rms=0.02, k_peak=3.0)
    f0 = orc.init(r, u, v)
    J, _, _ = forward_objective(spec, tau, F0, torch.from_numpy(f0).cuda())
    Jo = orc.objective(f0, tau, orc.Force(1, F0, 2, 1e-3), spec.n0, spec.n1, *spec.box, spec.L)
    assert abs(float(J) - Jo) < tol * abs(Jo), (float(J), Jo)


@pytest.mark.parametrize("n,box,L", [(32, (5, 3), 8), (32, (20, 27), 24), (6, (4, 5), 6)])
def test_gradients_match_oracle_finite_differences(P, orc, n, box, L):
    """dJ/dtau (h = 1e-6), dJ/dF0 (1e-3 relative step, Richardson) and a
    directional derivative in f0 against central differences of the FP64
    oracle objective; an 8 x 8 box and a 24 x 24 box on 32^2 (its stencil
    reach wraps onto the box: the adjoint's region is the whole grid), and
    the whole 6^2 grid as the box (the reach wraps around it twice)."""
    import dataclasses
    import torch
    from paper_1809_06735_gb300.adjoint import box_dissipation
    spec = dataclasses.replace(_small_spec(), nx=n, ny=n, box=box, L=L)
    tau0, kf, alpha = 0.6, 2, 1e-3
    F00 = li.kolmogorov_F0(n, tau0, kf, alpha, 0.02)
    r, u, v = li.random_phase(n, seed=4, u_rms=0.02, k_peak=3.0)
    f0 = orc.init(r, u, v)
    tau = torch.tensor(tau0, dtype=torch.float64, requires_grad=True)
    F0 = torch.tensor(F00, dtype=torch.float64, requires_grad=True)
    f0t = torch.from_numpy(f0).cuda().requires_grad_(True)
    J = box_dissipation(tau, F0, f0t, spec)
    J.backward()

    def Jo(t, a, f=f0):
        return orc.objective(f, t, orc.Force(1, a, kf, alpha), spec.n0, spec.n1, *spec.box,
                             spec.L)

    h = 1e-6
    fd_tau = (Jo(tau0 + h, F00) - Jo(tau0 - h, F00)) / (2 * h)
    assert abs(float(tau.grad) - fd_tau) < 1e-6 * abs(fd_tau)

    def dF(hr):
        a = F00 * hr
        return (Jo(tau0, F00 + a) - Jo(tau0, F00 - a)) / (2 * a)
    fd_F0 = (4 * dF(5e-4) - dF(1e-3)) / 3
    assert abs(float(F0.grad) - fd_F0) < 1e-6 * abs(fd_F0)

    rng = np.random.default_rng(9)
    d = rng.standard_normal(f0.shape) * 1e-3
    eps = 1e-4
    fd_f = (Jo(tau0, F00, f0 + eps * d) - Jo(tau0, F00, f0 - eps * d)) / (2 * eps)
    ad_f = float((f0t.grad.cpu().numpy() * d).sum())
    assert abs(ad_f - fd_f) < 1e-6 * abs(fd_f)


def test_fp32_forward_gradients_close_to_fp64(P):
    """The same gradients with the FP32 forward trajectory (adjoint in FP64)
    stay close to the FP64 ones over this short horizon."""
    import torch
    from paper_1809_06735_gb300.adjoint import box_dissipation
    r, u, v = li.random_phase(32, seed=4, u_rms=0.02, k_peak=3.0)
    import oracle
    f0 = torch.from_numpy(oracle.init(r, u, v)).cuda()
    F00 = li.kolmogorov_F0(32, 0.6, 2, 1e-3, 0.02)
    grads = []
    for prec in (64, 32):
        tau = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
        F0 = torch.tensor(F00, dtype=torch.float64, requires_grad=True)
        J = box_dissipation(tau, F0, f0, _small_spec(prec))
        J.backward()
        grads.append((float(tau.grad), float(F0.grad)))
    for a, b in zip(*grads):
        assert abs(a - b) < 1e-3 * abs(a)


# --------------------------------------------------------------------------
# The differentiation workload at its own configuration: 256^2, tau = 0.55,
# Kolmogorov forcing kf = 4 with drag 1e-4 and F0 for a laminar u_rms of
# 0.03, objective = mean over n in [1000, 2000] of the L = 16 box average
# (origin (0, 0)) of the dissipation term RHS^{E,4} of eq. (8), checkpoints
# every 100 steps, initial state from the random-phase generator (seed 0,
# u_rms 0.02).
# --------------------------------------------------------------------------

C3 = dict(n=256, tau=0.55, kf=4, alpha=1e-4, n0=1000, n1=2000, box=(0, 0), L=16, K=100)


def _c3_F0():
    return li.kolmogorov_F0(C3["n"], C3["tau"], C3["kf"], C3["alpha"], 0.03)


def _c3_oracle_J(args):
    """Oracle objective at (tau, F0) from the C3 initial state (one process)."""
    import oracle
    tau, F0 = args
    n = C3["n"]
    f0 = oracle.init(*li.random_phase(n, seed=0, u_rms=0.02))
    return oracle.objective(f0, tau, oracle.Force(1, F0, C3["kf"], C3["alpha"]), C3["n0"],
                            C3["n1"], *C3["box"], C3["L"])


@pytest.fixture(scope="module")
def c3_fd():
    """Oracle objective and its central finite differences: dJ/dtau with
    h = 1e-6, dJ/dF0 by Richardson extrapolation of central differences with
    relative steps 1e-3 and 5e-4 (seven oracle runs of 2000 steps, in
    parallel processes)."""
    import multiprocessing as mp
    tau, F0, h = C3["tau"], _c3_F0(), 1e-6
    pts = [(tau, F0), (tau + h, F0), (tau - h, F0)]
    for hr in (1e-3, 5e-4):
        pts += [(tau, F0 * (1 + hr)), (tau, F0 * (1 - hr))]
    with mp.get_context("spawn").Pool(len(pts)) as pool:
        v = pool.map(_c3_oracle_J, pts)
    d_tau = (v[1] - v[2]) / (2 * h)
    dF = [(v[3] - v[4]) / (2 * F0 * 1e-3), (v[5] - v[6]) / (2 * F0 * 5e-4)]
    return {"J": v[0], "dJ_dtau": d_tau, "dJ_dF0": (4 * dF[1] - dF[0]) / 3}


def _c3_gradients(P, precision):
    import torch
    from paper_1809_06735_gb300.adjoint import ObjectiveSpec, box_dissipation
    import oracle
    n = C3["n"]
    spec = ObjectiveSpec(nx=n, ny=n, kf=C3["kf"], alpha=C3["alpha"], n0=C3["n0"], n1=C3["n1"],
                         box=C3["box"], L=C3["L"], precision=precision,
                         checkpoint_every=C3["K"])
    f0 = torch.from_numpy(oracle.init(*li.random_phase(n, seed=0, u_rms=0.02))).cuda()
    tau = torch.tensor(C3["tau"], dtype=torch.float64, requires_grad=True)
    F0 = torch.tensor(_c3_F0(), dtype=torch.float64, requires_grad=True)
    J = box_dissipation(tau, F0, f0, spec)
    J.backward()
    return float(J.detach()), float(tau.grad), float(F0.grad)


@pytest.mark.slow
def test_c3_fp64_gradients_match_oracle_finite_differences(P, c3_fd):
    """FP64 forward, FP64 adjoint: J within 1e-10 of the oracle's (the FP64
    trajectories agree to rounding over the 2000 steps: the flow is not
    chaotic at this Reynolds number, the finite differences agree to 4e-10
    between h and 2h), dJ/dtau and dJ/dF0 within 1e-6 of the oracle's central
    finite differences."""
    J, gt, gF = _c3_gradients(P, 64)
    print("C3 FP64: J %.12e (oracle %.12e) dJ/dtau %.12e (FD %.12e) dJ/dF0 %.12e (FD %.12e)"
          % (J, c3_fd["J"], gt, c3_fd["dJ_dtau"], gF, c3_fd["dJ_dF0"]))
    assert abs(J - c3_fd["J"]) < 1e-10 * abs(c3_fd["J"])
    assert abs(gt - c3_fd["dJ_dtau"]) < 1e-6 * abs(c3_fd["dJ_dtau"])
    assert abs(gF - c3_fd["dJ_dF0"]) < 1e-6 * abs(c3_fd["dJ_dF0"])


@pytest.mark.slow
def test_c3_fp32_forward_gradients(P, c3_fd):
    """FP32 deviation forward, FP64 adjoint on its states: J and both
    gradients against the FP64 oracle's values.  The FP32 trajectory carries
    a relative population error of order 1e-6 per hundred steps (the step
    parity bar), so J (a sum of squared velocity gradients) and its
    derivatives differ from the FP64 values by the trajectory's relative
    error; bar 1e-4 over the 2000 steps."""
    J, gt, gF = _c3_gradients(P, 32)
    print("C3 FP32: J %.12e (oracle %.12e) dJ/dtau %.12e (FD %.12e) dJ/dF0 %.12e (FD %.12e)"
          % (J, c3_fd["J"], gt, c3_fd["dJ_dtau"], gF, c3_fd["dJ_dF0"]))
    assert abs(J - c3_fd["J"]) < 1e-4 * abs(c3_fd["J"])
    assert abs(gt - c3_fd["dJ_dtau"]) < 1e-4 * abs(c3_fd["dJ_dtau"])
    assert abs(gF - c3_fd["dJ_dF0"]) < 1e-4 * abs(c3_fd["dJ_dF0"])
