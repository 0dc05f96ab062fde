"""Full-size workloads on the GPU, checked where the oracle can follow them:
the forced tau-sweep (15 uneven members, 256^2..1024^2, one batched launch
per step) and the large 8192^2 forced run.  Sampled cells are compared with
the oracle's windowed run (exact inside the light cone of the window), the
whole grids with invariants that hold at any size.  Every oracle run starts
from the oracle's own initial state f_eq(rho, u) of the same host input
fields (the equilibrium is local, so a window of it is the equilibrium of
the window of the fields); nothing exported by the GPU enters the oracle."""
import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu
FP32_TOL = 2e-6
STEPS = 100  # the population parity horizon of the FP32 path


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def _windows_match(orc, fields, f_dev, n, steps, tau, force, points, half=8):
    """Compare (2 half) x (2 half) cells around each point after `steps`
    with the oracle's window run from the initial fields (rho, ux, uy)."""
    import torch
    w = 2 * half + 2 * steps
    for (px, py) in points:
        x0, y0 = (px - half - steps) % n, (py - half - steps) % n
        xi, yi = (x0 + np.arange(w)) % n, (y0 + np.arange(w)) % n
        win0 = orc.init(*(a[np.ix_(yi, xi)] for a in fields))
        xs = torch.tensor(xi, device=f_dev.device)
        ys = torch.tensor(yi, device=f_dev.device)
        got = f_dev.index_select(1, ys).index_select(2, xs).cpu().numpy()
        want = orc.run_window(win0, steps, tau, force, x0, y0, n, n)
        inner = (slice(None), slice(steps, w - steps), slice(steps, w - steps))
        err = np.max(np.abs(got[inner] - want[inner]) / np.abs(want[inner]))
        assert err < FP32_TOL, ((px, py), err)


def test_forced_tau_sweep_batched(P, orc):
    """15 members {256,512,1024}^2 x tau {0.505..0.6}, Kolmogorov kf = 4 with
    drag, in one batched launch per step, 100 steps: the 256^2 members
    against full oracle runs, the others on sampled windows; all members
    finite."""
    wl = li.forced_sweep_workload()
    mem = wl["members"]
    members = [P.Member(m["n"], m["n"], m["tau"], 1.0, 1, m["kf"], m["F0"], m["alpha"])
               for m in mem]
    lat = P.Lattice(members, precision=32, graph_steps=10)
    fields = []
    for i, m in enumerate(mem):
        fields.append(li.random_phase(m["n"], seed=m["seed"], u_rms=wl["u_rms"]))
        lat.init_fields(i, *fields[-1])
    lat.step(STEPS)
    rng = np.random.default_rng(3)
    for i, m in enumerate(mem):
        force = orc.Force(1, m["F0"], m["kf"], m["alpha"])
        f = lat.get_populations(i)
        assert lat.member_status(i) == 0
        if m["n"] == 256:
            ref = orc.run(orc.init(*fields[i]), STEPS, m["tau"], force)
            err = np.max(np.abs(f.cpu().numpy() - ref) / np.abs(ref))
            assert err < FP32_TOL, (i, err)
        else:
            pts = [tuple(p) for p in rng.integers(0, m["n"], size=(1, 2))] + [(0, 0)]
            _windows_match(orc, fields[i], f, m["n"], STEPS, m["tau"], force, pts)


def _large_fields(n, kmax=16):
    # smooth random initial fields (the spectral init of the workload needs
    # 8192^2 FFTs on the host; the step does not care which smooth field)
    r = 1.0 + li.smooth_fields(n, n, seed=7, amp=1e-3, kmax=kmax)
    u = li.smooth_fields(n, n, seed=5, amp=0.03, kmax=kmax)
    v = li.smooth_fields(n, n, seed=6, amp=0.03, kmax=kmax)
    return r, u, v


# The balance tests take modes up to |k| = 128 (wavelengths of 64 cells and
# more, the scales of the turbulent workloads' energy-containing range).
# With |k| <= 16 only, the third-derivative terms (RHS^{Omega,4},
# RHS^{Omega,5}) of an 8192^2 field are of order (2 pi 16 / 8192)^3 |u|,
# below what the rounding of |u| allows them to resolve (FP32: ~3e-2 of the
# field's magnitude; FP64: ~1e-9): an ill-conditioned input, not a test of
# the diagnostic.
BALANCE_KMAX = 128


def test_large_forced_8192_sampled(P, orc):
    """8192^2 forced run (tau 0.51, drag 1e-5), FP32: sampled windows against
    the oracle after 100 steps, and whole-grid mass conservation (FP32
    rounding of the collision is unbiased: ~2e-13 of the total over 67 M
    cells per step)."""
    import torch
    wl = li.large_forced_workload()
    n, tau = wl["n"], wl["tau"]
    m = P.Member(n, n, tau, 1.0, 1, wl["kf"], wl["F0"], wl["alpha"])
    lat = P.Lattice([m], precision=32, graph_steps=8)
    fields = _large_fields(n)
    lat.init_fields(0, *fields)
    g0 = lat.global_balance(0)
    lat.step(STEPS)
    g2 = lat.global_balance(0)
    f = lat.get_populations(0)
    force = orc.Force(1, wl["F0"], wl["kf"], wl["alpha"])
    pts = [(0, 0), (n - 1, n - 1), (4097, 123), (77, 8000)]
    _windows_match(orc, fields, f, n, STEPS, tau, force, pts)
    assert abs(g2[0] - g0[0]) < 1e-10 * g0[0]
    assert np.all(np.isfinite(g2))
    del f
    lat.close()
    torch.cuda.empty_cache()


def test_large_forced_8192_balance_identities(P):
    """One balance event of the 8192^2 FP32 member (the large-run
    configuration: FP32 deviation storage, FP32 term arithmetic, exact box
    sums, FP64 statistics) at every size of the workload, L = 2..4096, over
    all 67 M periodic origins, after 4 steps (time levels 2, 3, 4).  Two
    identities that hold at any size: the mean over all periodic origins of
    a box average is the grid mean of the field, so it is the same at every
    L; the divergence terms (RHS^{E,1}, RHS^{E,5}, RHS^{Omega,1},
    RHS^{Omega,5}) have a zero grid mean (periodic telescoping of eq. (18)).
    Bar 1e-4 of each term's spread over the L = 2 boxes."""
    import torch
    wl = li.large_forced_workload()
    n, tau, kf, F0, alpha, Ls = wl["n"], wl["tau"], wl["kf"], wl["F0"], wl["alpha"], wl["Ls"]
    lat = P.Lattice([P.Member(n, n, tau, 1.0, 1, kf, F0, alpha)], precision=32, diag_every=4)
    lat.init_fields(0, *_large_fields(n, BALANCE_KMAX))
    lat.step(4)
    stats = lat.subvolume_balance(0, Ls)
    lat.close()
    torch.cuda.empty_cache()
    assert np.all(np.isfinite(stats[:, 2:, :]))
    scale = np.abs(stats[0, 2:, 1]) + np.abs(stats[0, 2:, 0])
    for iL in range(len(Ls)):
        assert np.all(np.abs(stats[iL, 2:, 0] - stats[0, 2:, 0]) <= 1e-4 * scale), Ls[iL]
    for q in (3, 7, 9, 13):
        assert abs(stats[0, q, 0]) <= 1e-4 * scale[q - 2], q


@pytest.fixture(scope="module")
def window_terms(orc):
    """Oracle term fields of the 2048^2 window at the origin of the 8192^2
    forced run after 4 steps (levels 2, 3, 4), from the initial fields.  The
    window runs as its own periodic grid: 2048 divides 8192, so its
    Kolmogorov force with kf * 2048 / 8192 = 1 is the global force there,
    and a window cell is exact once it lies further from the window's edge
    than the 4 steps' light cone plus the 12 cells of the nested eq. (18)
    stencils (16 cells)."""
    wl = li.large_forced_workload()
    n, W = wl["n"], 2048
    fw = orc.Force(1, wl["F0"], wl["kf"] * W // n, wl["alpha"])
    f = orc.init(*(a[:W, :W] for a in _large_fields(n, BALANCE_KMAX)))
    f2 = orc.run(f, 2, wl["tau"], fw)
    f3 = orc.run(f2, 1, wl["tau"], fw)
    f4 = orc.run(f3, 1, wl["tau"], fw)
    return orc.terms_from_populations(f4, f3, f2, wl["tau"], fw)


@pytest.mark.slow
@pytest.mark.parametrize("dp,term_tol,delta_tol", [(64, 1e-10, 1e-6), (32, 1e-4, 1e-3)])
def test_large_grid_balance_boxes_match_the_oracle(P, orc, window_terms, dp, term_tol,
                                                   delta_tol):
    """The balance event on the 8192^2 grid (tables and scratch sized for
    67 M cells) per box against the oracle, for L = 2..1024 on 24 boxes per
    size inside the 2048^2 window (16 cells from its edges).  FP64
    populations, so the GPU and oracle trajectories agree to rounding and
    the comparison isolates the diagnostic; term arithmetic in FP64
    (dp = 64: terms within 1e-10 of each field's magnitude, as the other
    FP64 diagnostic tests) and in FP32 (dp = 32, the large run's arithmetic:
    1e-4).  A balancing error divides a cancelling sum by the box's
    max |RHS|, so with FP64 terms its error is bounded by the terms' bar
    propagated through that quotient: term_tol * (sum of the balance's
    field magnitudes) / max |RHS| (times 2 for the quotient's two
    roundings), checked per box; with FP32 terms, the mean over each size's
    boxes within 1e-3 relative (the bar of the FP32 balancing-error
    statistics)."""
    import torch
    wl = li.large_forced_workload()
    n, tau, kf, F0, alpha = wl["n"], wl["tau"], wl["kf"], wl["F0"], wl["alpha"]
    W, margin = 2048, 16
    Lw = [L for L in wl["Ls"] if L <= 1024]
    rng = np.random.default_rng(17)
    origins = [rng.integers(margin, W - margin - L + 1, size=(24, 2)) for L in Lw]
    lat = P.Lattice([P.Member(n, n, tau, 1.0, 1, kf, F0, alpha)], precision=64, diag_every=4,
                    diag_precision=dp)
    lat.init_fields(0, *_large_fields(n, BALANCE_KMAX))
    lat.step(4)
    _, pb = lat.subvolume_balance(0, Lw, origins=origins, per_box=True)
    pb = pb.cpu().numpy()
    lat.close()
    torch.cuda.empty_cache()
    T = window_terms
    inner = (slice(None), slice(margin, W - margin), slice(margin, W - margin))
    term_scale = np.max(np.abs(T[inner].reshape(13, -1)), axis=1) + 1e-300
    row, worst = 0, 0.0
    for iL, L in enumerate(Lw):
        dg, dw = [], []
        for (x0, y0) in origins[iL]:
            want = orc.box_values(T, x0, y0, L)
            got = pb[row]
            row += 1
            d = np.abs(got[2:] - want[2:]) / term_scale
            worst = max(worst, float(np.max(d)))
            assert np.max(d) < term_tol, (L, x0, y0, int(np.argmax(d)), float(np.max(d)))
            if dp == 64:
                for q, (lo, hi) in enumerate(((0, 6), (6, 13))):  # energy, enstrophy
                    rhs = np.max(np.abs(want[2 + lo + 1:2 + hi]))
                    bound = 2 * term_tol * np.sum(term_scale[lo:hi]) / rhs * max(1.0, want[q])
                    assert abs(got[q] - want[q]) <= bound, (L, x0, y0, q, got[q], want[q], bound)
            dg.append(got[:2])
            dw.append(want[:2])
        mg, mw = np.mean(dg, axis=0), np.mean(dw, axis=0)
        assert np.all(np.abs(mg - mw) <= delta_tol * np.abs(mw) + 1e-12), (L, mg, mw)
    assert row == pb.shape[0]
    print("8192^2 boxes, term arithmetic FP%d: worst term error %.2e of the field's magnitude"
          % (dp, worst))
