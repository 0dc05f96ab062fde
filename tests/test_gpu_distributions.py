"""GPU parity of the distributions over boxes (the PDFs of the balancing
errors shown in Sec. 4 and the sub-volume Mach number of eq. (20)) against
the FP64 oracle, through the C ABI.

Histogram counts are integers: a box whose value lies within the rounding
of the two sides' evaluations (1e-9 relative for the FP64 diagnostic, whose
box terms agree with the oracle to 1e-10 of each field's magnitude) of a bin
edge may land on either side of it; every other box must land in the same
bin.  The test counts the oracle's boxes inside that zone and allows at most
that many moves."""
import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu

DELTA_EDGES = np.geomspace(1e-9, 10.0, 41)
MACH_EDGES = np.linspace(0.0, 0.12, 25)


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def _box_list(nx, ny, origins):
    if origins is None:
        return [(b % nx, b // nx) for b in range(nx * ny)]
    return [tuple(int(v) for v in o) for o in origins]


def _near_edge(v, edges, rel):
    v = np.asarray(v, dtype=float)
    e = np.asarray(edges)[None, :]
    zone = rel * np.maximum(np.abs(e), np.abs(v)[:, None]) + 1e-300
    return np.any(np.abs(v[:, None] - e) <= zone, axis=1)


def _check_hist(got, want, ambiguous):
    assert got.sum() == want.sum()
    assert np.abs(got - want).sum() <= 2 * ambiguous, (got, want, ambiguous)


def _oracle_case(orc, T, ux, uy, Ls, origins, nx, ny):
    hd, hm, ms = orc.distributions(T, ux, uy, Ls, DELTA_EDGES, MACH_EDGES, origins=origins)
    _, pb = orc.balance_stats(T, Ls, origins=origins, per_box=True)
    boxes = _box_list(nx, ny, origins)
    mach = np.array([[orc.box_mach(ux, uy, x0, y0, L) for (x0, y0) in boxes] for L in Ls])
    return hd, hm, ms, pb, mach


@pytest.mark.parametrize("origin_mode", ["all", "list"])
def test_distributions_fp64_against_oracle(P, orc, origin_mode):
    """Forced flow on a 56 x 40 grid (FP64): Ma_V statistics within 1e-10 of
    the oracle, histogram counts equal up to boxes at an edge, the balance
    statistics equal to the plain balance call, L > N rows empty."""
    nx, ny, tau = 56, 40, 0.53
    force = orc.Force(1, 3e-4, 2, 1e-3)
    lat = P.Lattice([P.Member(nx, ny, tau, 1.0, 1, 2, 3e-4, 1e-3)], precision=64)
    r = 1.0 + li.smooth_fields(nx, ny, 40, amp=0.01)
    u = li.smooth_fields(nx, ny, 41, amp=0.03)
    v = li.smooth_fields(nx, ny, 42, amp=0.03)
    lat.init_fields(0, r, u, v)
    lat.step(30)
    lat.record_snapshot()
    f30 = lat.get_populations_host(0)
    lat.step(1)
    lat.record_snapshot()
    f31 = lat.get_populations_host(0)
    lat.step(1)
    f32 = lat.get_populations_host(0)
    Ls = [1, 4, 13, 40, 41]
    origins = None
    if origin_mode == "list":
        origins = np.stack([np.arange(300) % nx, (np.arange(300) * 7) % ny], 1).astype(np.int32)
    got = lat.subvolume_distributions([0], Ls, DELTA_EDGES, MACH_EDGES, origins=origins)
    plain = lat.subvolume_balance(0, Ls, origins=origins)
    np.testing.assert_allclose(got["stats"][0], plain, rtol=1e-13, atol=1e-300)
    T = orc.terms_from_populations(f32, f31, f30, tau, force)
    m = orc.moments(f32, force)
    ux, uy = m["ux"], m["uy"]
    fit = [i for i, L in enumerate(Ls) if L <= min(nx, ny)]
    hd, hm, ms, pb, mach = _oracle_case(orc, T, ux, uy, [Ls[i] for i in fit], origins, nx, ny)
    for k, iL in enumerate(fit):
        np.testing.assert_allclose(got["mach"][0, iL], ms[k], rtol=1e-10, atol=1e-14)
        for q in range(2):
            amb = int(_near_edge(pb[k][:, q], DELTA_EDGES, 1e-9).sum())
            _check_hist(got["delta_hist"][0, iL, q], hd[k, q], amb)
        amb = int(_near_edge(mach[k], MACH_EDGES, 1e-9).sum())
        _check_hist(got["mach_hist"][0, iL], hm[k], amb)
    for iL in range(len(Ls)):
        if iL not in fit:
            assert got["delta_hist"][0, iL].sum() == 0 and got["mach_hist"][0, iL].sum() == 0
            assert np.all(np.isnan(got["mach"][0, iL]))


def test_distributions_fp32_ensemble_and_batching(P, orc):
    """Uneven FP32 members (FP32 diagnostic): every box counted once per
    size, Ma_V statistics within 1e-5 of the oracle's on the exported states,
    Ma_V histograms equal up to boxes within 1e-5 of an edge, and results
    independent of how many members share a launch."""
    spec = [(48, 40, 0.55), (64, 64, 0.6), (37, 23, 0.52)]
    Ls = [2, 8, 23, 40]
    res = []
    states = []
    for batch in (1, 0):
        lat = P.Lattice([P.Member(nx, ny, t) for nx, ny, t in spec], precision=32,
                        diag_every=16, diag_batch=batch)
        for i, (nx, ny, _) in enumerate(spec):
            lat.init_fields(i, 1.0 + li.smooth_fields(nx, ny, 50 + i, amp=0.01),
                            li.smooth_fields(nx, ny, 60 + i, amp=0.04),
                            li.smooth_fields(nx, ny, 70 + i, amp=0.04))
        lat.step(16)
        res.append(lat.subvolume_distributions(range(3), Ls, DELTA_EDGES, MACH_EDGES))
        states = [lat.get_populations_host(i) for i in range(3)]
    for key in ("delta_hist", "mach_hist"):
        np.testing.assert_array_equal(res[0][key], res[1][key])
    np.testing.assert_array_equal(res[0]["mach"], res[1]["mach"])
    got = res[1]
    for i, (nx, ny, _) in enumerate(spec):
        m = orc.moments(states[i])
        ux, uy = m["ux"], m["uy"]
        for iL, L in enumerate(Ls):
            if L > min(nx, ny):
                assert got["mach_hist"][i, iL].sum() == 0
                assert np.all(np.isnan(got["mach"][i, iL]))
                continue
            assert got["delta_hist"][i, iL, 0].sum() == nx * ny
            assert got["delta_hist"][i, iL, 1].sum() == nx * ny
            mach = np.array([orc.box_mach(ux, uy, x0, y0, L) for (x0, y0) in _box_list(nx, ny, None)])
            np.testing.assert_allclose(got["mach"][i, iL, 0], mach.mean(), rtol=1e-5)
            np.testing.assert_allclose(got["mach"][i, iL, 1], mach.std(), rtol=2e-3,
                                       atol=1e-5 * mach.mean())
            want = np.bincount(np.searchsorted(MACH_EDGES, mach, side="right"),
                               minlength=len(MACH_EDGES) + 1)
            amb = int(_near_edge(mach, MACH_EDGES, 1e-5).sum())
            _check_hist(got["mach_hist"][i, iL], want, amb)


def test_distributions_full_size_table1(P, orc):
    """One 512^2 member of the decaying ensemble (FP32 populations, FP64
    diagnostic) on the paper's Table 1 random boxes at L = 2, 16, 128, 256:
    counts and Ma_V statistics against the oracle on the exported states."""
    wl = li.decaying_ensemble_workload(members=1)
    n, tau = wl["n"], wl["tau"]
    lat = P.Lattice([P.Member(n, n, tau)], precision=32, diag_precision=64)
    lat.init_fields(0, *li.random_phase(n, seed=1000, u_rms=wl["u_rms"]))
    lat.step(40)
    lat.record_snapshot()
    f40 = lat.get_populations_host(0)
    lat.step(1)
    lat.record_snapshot()
    f41 = lat.get_populations_host(0)
    lat.step(1)
    f42 = lat.get_populations_host(0)
    Ls = [2, 16, 128, 256]
    origins = [li.table1_origins(n, L, seed=7 + L) for L in Ls]
    got = lat.subvolume_distributions([0], Ls, DELTA_EDGES, MACH_EDGES, origins=origins)
    T = orc.terms_from_populations(f42, f41, f40, tau)
    m = orc.moments(f42)
    ux, uy = m["ux"], m["uy"]
    for iL, L in enumerate(Ls):
        hd, hm, ms = orc.distributions(T, ux, uy, [L], DELTA_EDGES, MACH_EDGES,
                                       origins=origins[iL])
        _, pb = orc.balance_stats(T, [L], origins=origins[iL], per_box=True)
        mach = np.array([orc.box_mach(ux, uy, x0, y0, L) for (x0, y0) in origins[iL]])
        np.testing.assert_allclose(got["mach"][0, iL], ms[0], rtol=1e-9, atol=1e-14)
        for q in range(2):
            amb = int(_near_edge(pb[0][:, q], DELTA_EDGES, 1e-7).sum())
            _check_hist(got["delta_hist"][0, iL, q], hd[0, q], amb)
        _check_hist(got["mach_hist"][0, iL], hm[0], int(_near_edge(mach, MACH_EDGES, 1e-9).sum()))


def test_distributions_rejects_bad_edges(P):
    n = 16
    lat = P.Lattice([P.Member(n, n, 0.6)], precision=64, diag_every=4)
    lat.init_fields(0, np.ones((n, n)), li.smooth_fields(n, n, 1), li.smooth_fields(n, n, 2))
    lat.step(4)
    for de in ([], [1.0, 1.0], [2.0, 1.0], [0.0, np.inf], list(np.linspace(0, 1, 257))):
        with pytest.raises(P.LBMError) as e:
            lat.subvolume_distributions([0], [4], de, MACH_EDGES)
        assert e.value.code == -1
    ok = lat.subvolume_distributions([0], [4], [0.5], [0.01])
    assert ok["delta_hist"].shape == (1, 1, 2, 2) and ok["mach_hist"].shape == (1, 1, 2)
