"""GPU parity of the diagnostic (moments, whole-grid budget, sub-volume
balance terms, balancing errors and their statistics: eqs. (8)-(13), (17),
(18), Table 1) against the FP64 oracle, through the C ABI."""
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


def _forced_state(orc, nx, ny, tau, force, steps, seed):
    r = 1.0 + li.smooth_fields(nx, ny, seed, amp=0.01)
    u = li.smooth_fields(nx, ny, seed + 1, amp=0.03)
    v = li.smooth_fields(nx, ny, seed + 2, amp=0.03)
    return (r, u, v), orc.run(orc.init(r, u, v), steps, tau, force)


def test_moments_and_vorticity(P, orc):
    nx, ny, tau = 48, 40, 0.55
    force = orc.Force(1, 2e-4, 3, 5e-3)
    _, f = _forced_state(orc, nx, ny, tau, force, 0, 20)
    lat = P.Lattice([P.Member(nx, ny, tau, 1.0, 1, 3, 2e-4, 5e-3)], precision=64)
    lat.set_populations(0, f)
    got = {k: v.cpu().numpy() for k, v in lat.moments(0).items()}
    m = orc.moments(f, force)
    w = orc.ddx(m["uy"]) - orc.ddy(m["ux"])
    for k, ref in (("rho", m["rho"]), ("ux", m["ux"]), ("uy", m["uy"]), ("omega", w)):
        assert np.max(np.abs(got[k] - ref)) <= 1e-13 * np.max(np.abs(ref)), k


@pytest.mark.parametrize("prec", [64, 32])
def test_global_balance(P, orc, prec):
    nx, ny, tau = 64, 48, 0.6
    force = orc.Force(1, 1e-4, 2, 1e-4)
    _, f = _forced_state(orc, nx, ny, tau, force, 0, 30)
    lat = P.Lattice([P.Member(nx, ny, tau, 1.0, 1, 2, 1e-4, 1e-4)], precision=prec)
    lat.set_populations(0, f)
    got = lat.global_balance(0)
    ref = orc.global_quantities(lat.get_populations_host(0), tau, force)
    np.testing.assert_allclose(got[[0, 3, 4, 5, 6]], ref[[0, 3, 4, 5, 6]], rtol=1e-12)
    assert abs(got[1] - ref[1]) < 1e-12 * nx * ny and abs(got[2] - ref[2]) < 1e-12 * nx * ny


# FP64 tolerance of the box terms, relative to each term field's largest
# magnitude.  Both sides round differently (stencil pairing, SAT versus brute
# force sums); the worst-conditioned term is RHS^{E,2} = -u . grad p with
# p = rho/3: rho varies by ~1e-4 around 1, so the eq. (18) difference of p
# cancels ~|p|/|grad p| ~ 1e5 and one-ulp input differences reach ~1e-11
# of the term.  1e-10 keeps a 10x margin and still fails any wrong sign,
# index, missing factor or FP32 leak (>= 1e-7).
TERM_TOL = 1e-10
DELTA_TOL = 1e-8


def _check_boxes(got_stats, got_pb, T, Ls, origins=None):
    import oracle as orc
    want, want_pb = orc.balance_stats(T, Ls, origins=origins, per_box=True)
    term_scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
    worst = 0.0
    for iL in range(len(Ls)):
        # terms: relative to the field's magnitude
        d = np.abs(got_pb[iL][:, 2:] - want_pb[iL][:, 2:]) / term_scale[None, :]
        worst = max(worst, float(np.max(d)))
        assert np.max(d) < TERM_TOL, (Ls[iL], np.argmax(np.max(d, axis=0)), np.max(d))
        # balancing errors: they divide a cancelling sum by max |RHS|
        dd = np.abs(got_pb[iL][:, :2] - want_pb[iL][:, :2])
        assert np.max(dd) < DELTA_TOL * max(1.0, np.max(want_pb[iL][:, :2])), Ls[iL]
        np.testing.assert_allclose(got_stats[iL, 2:, 0], want[iL, 2:, 0],
                                   rtol=0, atol=TERM_TOL * np.max(term_scale))
        np.testing.assert_allclose(got_stats[iL, 2:, 1], want[iL, 2:, 1], rtol=1e-7,
                                   atol=TERM_TOL * np.max(term_scale))
        np.testing.assert_allclose(got_stats[iL, :2, :], want[iL, :2, :], rtol=1e-6,
                                   atol=DELTA_TOL)
    return worst


def test_balance_taylor_green_64_fp64(P, orc):
    """Plain FP64 Taylor-Green at 64^2, every periodic origin, L in {4,8,16,32}
    at step 100 (diagnostic history 98, 99, 100).  The diagnostic is compared
    on the GPU's own exported states (the BDF2 time derivative cancels about
    three digits, so trajectory rounding differences must not enter); the
    trajectory itself is checked against the oracle separately."""
    wl = li.taylor_green_workload()
    n, tau = wl["n"], wl["tau"]
    rho, ux, uy = li.taylor_green(n, u0=wl["u0"])
    lat = P.Lattice([P.Member(n, n, tau)], precision=64, diag_every=wl["diag_every"])
    lat.init_fields(0, rho, ux, uy)
    lat.step(98)
    f98 = lat.get_populations_host(0)
    lat.step(1)
    f99 = lat.get_populations_host(0)
    lat.step(1)
    f100 = lat.get_populations_host(0)
    stats, pb = lat.subvolume_balance(0, wl["Ls"], per_box=True)
    ref100 = orc.run(orc.init(rho, ux, uy), 100, tau)
    assert np.max(np.abs(f100 - ref100) / ref100) < 1e-12
    T = orc.terms_from_populations(f100, f99, f98, tau)
    worst = _check_boxes(stats, pb.cpu().numpy().reshape(len(wl["Ls"]), -1, 15), T, wl["Ls"])
    print("64^2 Taylor-Green, FP64 terms: worst per-box term error %.2e of the field's magnitude"
          % worst)


def test_balance_forced_ragged_origin_list(P, orc):
    """Forced flow on a non-square grid, Table 1 random origins, sizes beyond
    the grid skipped (NaN), FP64."""
    nx, ny, tau = 56, 40, 0.53
    force = orc.Force(1, 3e-4, 2, 1e-3)
    lat = P.Lattice([P.Member(nx, ny, tau, 1.0, 1, 2, 3e-4, 1e-3)], precision=64)
    (r, u, v), _ = _forced_state(orc, nx, ny, tau, force, 0, 40)
    lat.init_fields(0, r, u, v)
    lat.step(30)
    lat.record_snapshot()
    f30 = lat.get_populations_host(0)
    lat.step(1)
    lat.record_snapshot()
    f31 = lat.get_populations_host(0)
    lat.step(1)
    f32 = lat.get_populations_host(0)
    origins = np.stack([np.arange(0, 300) % nx, (np.arange(0, 300) * 7) % ny], 1).astype(np.int32)
    Ls = [1, 3, 7, 16, 40, 41, 64]
    stats = lat.subvolume_balance(0, Ls, origins=origins)
    assert np.all(np.isnan(stats[5:]))
    stats_v, pb = lat.subvolume_balance(0, Ls[:5], origins=origins, per_box=True)
    np.testing.assert_array_equal(stats[:5], stats_v)
    T = orc.terms_from_populations(f32, f31, f30, tau, force)
    _check_boxes(stats_v, pb.cpu().numpy().reshape(5, -1, 15), T, Ls[:5], origins=origins)


def test_balance_history_required(P):
    n = 16
    lat = P.Lattice([P.Member(n, n, 0.6)], precision=64)
    lat.init_fields(0, np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)))
    lat.step(5)
    with pytest.raises(P.LBMError) as e:
        lat.subvolume_balance(0, [4])
    assert e.value.code == -4


def test_balance_fp32_against_fp64_oracle(P, orc):
    """FP32 deviation populations feeding the FP64 diagnostic: the box terms
    stay within 1e-4 relative (of each term's magnitude) of the FP64 oracle
    over a 100-step horizon."""
    n, tau = 64, 0.55
    force = orc.Force(1, li.kolmogorov_F0(n, tau, 4, 1e-4, 0.03), 4, 1e-4)
    rho, ux, uy = li.random_phase(n, seed=5, u_rms=0.02)
    lat = P.Lattice([P.Member(n, n, tau, 1.0, 1, 4, force.F0, 1e-4)], precision=32,
                    diag_every=100)
    lat.init_fields(0, rho, ux, uy)
    lat.step(100)
    Ls = [2, 4, 8, 16, 32, 64]
    stats, pb = lat.subvolume_balance(0, Ls, per_box=True)
    pb = pb.reshape(len(Ls), n * n, 15)
    f98 = orc.run(orc.init(rho, ux, uy), 98, tau, force)
    f99 = orc.run(f98, 1, tau, force)
    f100 = orc.run(f99, 1, tau, force)
    T = orc.terms_from_populations(f100, f99, f98, tau, force)
    want, want_pb = orc.balance_stats(T, Ls, per_box=True)
    pb = pb.cpu().numpy()
    scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
    for iL in range(len(Ls)):
        d = np.abs(pb[iL][:, 2:] - want_pb[iL][:, 2:]) / scale[None, :]
        assert np.max(d) < 1e-4, (Ls[iL], np.max(d))


def test_balance_full_size_sampled(P, orc):
    """One 512^2 member at the ensemble's box sizes L = 2..256, all origins on
    the GPU; sampled boxes against the oracle's brute-force averages of the
    oracle terms of the same exported states; the all-origin mean of every
    term equals its global mean."""
    wl = li.decaying_ensemble_workload(members=2)
    n, tau = wl["n"], wl["tau"]
    for diag_prec, term_tol in ((64, TERM_TOL), (32, FP32_TERM_TOL)):
        lat = P.Lattice([P.Member(n, n, tau)] * 2, precision=32, diag_every=wl["diag_every"],
                        graph_steps=20, diag_precision=diag_prec)
        for m in range(2):
            lat.init_fields(m, *li.random_phase(n, seed=wl["seed0"] + m, u_rms=wl["u_rms"]))
        lat.step(198)
        f198 = lat.get_populations_host(1)
        lat.step(1)
        f199 = lat.get_populations_host(1)
        lat.step(1)
        f200 = lat.get_populations_host(1)
        stats, pb = lat.subvolume_balance(1, wl["Ls"], per_box=True)
        T = orc.terms_from_populations(f200, f199, f198, tau)
        rng = np.random.default_rng(0)
        idx = rng.integers(0, n * n, size=40)
        pb = pb.cpu().numpy().reshape(len(wl["Ls"]), n * n, 15)
        scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
        for iL, L in enumerate(wl["Ls"]):
            for b in idx:
                want = orc.box_values(T, b % n, b // n, L)
                err = np.max(np.abs(pb[iL, b, 2:] - want[2:]) / scale)
                assert err < term_tol, (diag_prec, L, err)
                if diag_prec == 64:
                    assert abs(pb[iL, b, 0] - want[0]) < DELTA_TOL
                    assert abs(pb[iL, b, 1] - want[1]) < DELTA_TOL
            np.testing.assert_allclose(stats[iL, 2:, 0], T.reshape(13, -1).mean(axis=1),
                                       rtol=0, atol=term_tol * np.max(scale))
        lat.close()


# FP32 diagnostic arithmetic: term fields from FP32 stencils on FP32
# velocities whose level differences are formed in FP64.  The relative FP32
# rounding (6e-8) is amplified by each eq. (18) difference by about
# |A| / |D A| (~10 at the energetic scales of these grids); the enstrophy
# terms RHS^{O,4}, RHS^{O,5} nest three differences (w, H = D(nu rho S), then
# D(w H)), so their error reaches ~6e-5 of the field's magnitude (measured
# 4.4e-5 and 6.0e-5 on the 256^2 and 512^2 workloads).  The bar is the 1e-4
# relative tolerance on FP32 balance terms.
FP32_TERM_TOL = 1e-4


def test_balance_fp32_diagnostic_table1_origins(P, orc):
    """FP32 handle with its default FP32 diagnostic on the paper's Table 1
    random boxes (a different box list per size): per-box terms within the
    FP32 tolerance, balancing-error statistics within 1e-3 relative, of the
    oracle on the same exported states."""
    n, tau = 256, 0.55
    F0 = li.kolmogorov_F0(n, tau, 4, 1e-4, 0.03)
    force = orc.Force(1, F0, 4, 1e-4)
    lat = P.Lattice([P.Member(n, n, tau, 1.0, 1, 4, F0, 1e-4)], precision=32, diag_every=50)
    lat.init_fields(0, *li.random_phase(n, seed=77, u_rms=0.03))
    lat.step(48)
    f48 = lat.get_populations_host(0)
    lat.step(1)
    f49 = lat.get_populations_host(0)
    lat.step(1)
    f50 = lat.get_populations_host(0)
    Ls = [2, 8, 32, 100, 181, 256]
    origins = [li.table1_origins(n, L, seed=L) for L in Ls]
    stats, pb = lat.subvolume_balance(0, Ls, origins=origins, per_box=True)
    pb = pb.cpu().numpy()
    T = orc.terms_from_populations(f50, f49, f48, tau, force)
    scale = np.max(np.abs(T.reshape(13, -1)), axis=1) + 1e-300
    row = 0
    for iL, L in enumerate(Ls):
        o = origins[iL]
        assert o.shape[0] == li.table1_count(L, n)
        want, want_pb = orc.balance_stats(T, [L], origins=o, per_box=True)
        got = pb[row:row + o.shape[0]]
        row += o.shape[0]
        err = np.max(np.abs(got[:, 2:] - want_pb[0][:, 2:]) / scale[None, :])
        assert err < FP32_TERM_TOL, (L, err)
        np.testing.assert_allclose(stats[iL, :2, 0], want[0, :2, 0], rtol=1e-3)
        np.testing.assert_allclose(stats[iL, 2:, 0], want[0, 2:, 0], rtol=0,
                                   atol=FP32_TERM_TOL * np.max(scale))
    assert row == pb.shape[0]


def test_balance_batch_equals_per_member(P):
    """The batched call over uneven members gives, bit for bit, the per-member
    statistics; sizes beyond a member's grid are NaN for that member only."""
    spec = [(32, 32, 0.6), (48, 40, 0.55), (64, 64, 0.52)]
    lat = P.Lattice([P.Member(nx, ny, t) for nx, ny, t in spec], precision=32, diag_every=20)
    for i, (nx, ny, _) in enumerate(spec):
        u = li.smooth_fields(nx, ny, 50 + i, amp=0.03)
        v = li.smooth_fields(nx, ny, 60 + i, amp=0.03)
        lat.init_fields(i, np.ones((ny, nx)), u, v)
    lat.step(20)
    Ls = [2, 8, 32, 40, 64]
    batch = lat.subvolume_balance_batch([0, 1, 2], Ls)
    for i in range(3):
        single = lat.subvolume_balance(i, Ls)
        np.testing.assert_array_equal(batch[i], single)
    # 32x32 fits L <= 32; 48x40 fits L <= 40; 64x64 fits every size
    assert np.all(np.isnan(batch[0, 3:])) and np.all(np.isfinite(batch[0, :3, 2:, 0]))
    assert np.all(np.isnan(batch[1, 4:])) and np.all(np.isfinite(batch[1, :4, 2:, 0]))
    assert np.all(np.isfinite(batch[2, :, 2:, 0]))


def test_async_balance_overlapped_with_stepping(P):
    """The asynchronous diagnostic gives, bit for bit, the synchronous
    statistics of the same time even while the next steps run on the main
    stream; the next snapshot records wait for it."""
    import torch
    spec = [(64, 64, 0.55), (48, 40, 0.6), (128, 32, 0.52)]
    lat = P.Lattice([P.Member(nx, ny, t) for nx, ny, t in spec], precision=32, diag_every=20,
                    graph_steps=6)
    for i, (nx, ny, _) in enumerate(spec):
        lat.init_fields(i, 1.0 + li.smooth_fields(nx, ny, 70 + i, amp=0.01),
                        li.smooth_fields(nx, ny, 80 + i, amp=0.03),
                        li.smooth_fields(nx, ny, 90 + i, amp=0.03))
    lat.step(20)
    Ls = [2, 4, 16, 40]
    origins = [li.table1_origins(32, L, seed=L, count=500) for L in (2, 4, 16)] + \
        [np.zeros((1, 2), np.int32)]
    ref = lat.subvolume_balance_batch([0, 1, 2], Ls, origins=origins)
    out = lat.subvolume_balance_async([0, 1, 2], Ls, origins=origins)
    lat.step(15)
    lat.diag_synchronize()
    got = out.cpu().numpy()
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    np.testing.assert_array_equal(got[~np.isnan(got)], ref[~np.isnan(ref)])
    lat.step(5)  # records 38, 39, 40 after the asynchronous work
    nxt = lat.subvolume_balance_batch([0, 1, 2], Ls, origins=origins)
    assert np.all(np.isfinite(nxt[:, :3, 2:, 0]))
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", [32, 64])
def test_batched_diagnostic_independent_of_batch_size(P, prec):
    """One member per diagnostic launch, two per launch (three batches, slots
    reused) and all in one launch give bit-identical statistics, for uneven
    grids with ragged 32 x 8 cell tiles, all periodic origins and origin
    lists."""
    spec = [(37, 23, 0.6), (64, 48, 0.55), (8, 8, 0.7), (130, 20, 0.52), (64, 48, 0.58)]
    Ls = [2, 5, 8, 20, 40]
    # origins inside the smallest grid (8 x 8) for L <= 8; the origin (0, 0)
    # for the larger sizes
    origins = [li.table1_origins(8, L, seed=L, count=300) if L <= 8 else
               np.zeros((3, 2), np.int32) for L in Ls]
    res = []
    for batch in (1, 2, 0):
        lat = P.Lattice([P.Member(nx, ny, t) for nx, ny, t in spec], precision=prec,
                        diag_every=12, diag_batch=batch)
        for i, (nx, ny, _) in enumerate(spec):
            lat.init_fields(i, 1.0 + li.smooth_fields(nx, ny, 10 + i, amp=0.01),
                            li.smooth_fields(nx, ny, 20 + i, amp=0.03),
                            li.smooth_fields(nx, ny, 30 + i, amp=0.03))
        lat.step(12)
        res.append((lat.subvolume_balance_batch(range(len(spec)), Ls),
                    lat.subvolume_balance_batch(range(len(spec)), Ls, origins=origins)))
    for a, b in res[1:]:
        for x, y in ((res[0][0], a), (res[0][1], b)):
            np.testing.assert_array_equal(np.isnan(x), np.isnan(y))
            np.testing.assert_array_equal(x[~np.isnan(x)], y[~np.isnan(y)])
    # sizes that fit: 8x8 only L <= 8; 130x20 and 37x23 L <= 20
    assert np.all(np.isnan(res[0][0][2, 3:])) and np.all(np.isfinite(res[0][0][2, :3, 2:, 0]))
    assert np.all(np.isfinite(res[0][0][1, :, 2:, 0]))
