"""GPU parity of the D2Q9 stream-collide (eq. (1), eq. (2), EDM forcing)
against the FP64 oracle, through the C ABI.

Bars: FP64 path within 1e-12 relative on every population; FP32 deviation
path within 2e-6 relative on the full populations over 100 steps; state
conversion bit-exact where it is a permutation.
"""
import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-6


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def rel_err(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


def _fields(nx, ny, seed, amp=0.03):
    u = li.smooth_fields(nx, ny, seed, amp=amp)
    v = li.smooth_fields(nx, ny, seed + 1, amp=amp)
    r = 1.0 + li.smooth_fields(nx, ny, seed + 2, amp=0.01)
    return r, u, v


def test_fp64_taylor_green_64_parity(P, orc):
    """Plain FP64 Taylor-Green 64^2, tau 0.6, 1000 steps."""
    wl = li.taylor_green_workload()
    n, tau = wl["n"], wl["tau"]
    rho, ux, uy = li.taylor_green(n, u0=wl["u0"])
    lat = P.Lattice([P.Member(n, n, tau)], precision=64, graph_steps=16)
    lat.init_fields(0, rho, ux, uy)
    lat.step(wl["steps"])
    assert lat.time == wl["steps"]
    ref = orc.run(orc.init(rho, ux, uy), wl["steps"], tau)
    assert rel_err(lat.get_populations_host(0), ref) < FP64_TOL


def test_fp64_ragged_forced_random_state(P, orc):
    """Non-square ragged grid, random populations, Kolmogorov force + drag:
    every population lands on its cell (index placement) to FP64 rounding."""
    nx, ny, tau = 37, 23, 0.53
    m = P.Member(nx, ny, tau, 1.0, 1, 2, 3e-4, 2e-3)
    f0 = li.random_populations(nx, ny, seed=11)
    lat = P.Lattice([m], precision=64)
    lat.set_populations(0, f0)
    lat.step(60)
    ref = orc.run(f0, 60, tau, orc.Force(1, 3e-4, 2, 2e-3))
    assert rel_err(lat.get_populations_host(0), ref) < FP64_TOL


def _batch_members():
    return [
        (136, 40, 0.52, 1, 2, 1e-4, 1e-4),   # x tail past one 128-cell warp row
        (256, 64, 0.6, 0, 0, 0.0, 0.0),
        (64, 30, 0.55, 1, 1, 2e-5, 0.0),
        (132, 17, 0.51, 0, 0, 0.0, 1e-3),
    ]


@pytest.mark.parametrize("graph_steps", [0, 16])
def test_fp32_batched_parity(P, orc, graph_steps):
    """Uneven members in one batched launch, 100 steps, FP32 deviation form."""
    spec = _batch_members()
    members = [P.Member(nx, ny, tau, 1.0, fk, 4, F0, a) for (nx, ny, tau, fk, _, F0, a) in spec]
    lat = P.Lattice(members, precision=32, graph_steps=graph_steps)
    inits = []
    for i, (nx, ny, *_r) in enumerate(spec):
        r, u, v = _fields(nx, ny, 100 + 3 * i)
        lat.init_fields(i, r, u, v)
        inits.append((r, u, v))
    lat.step(100)
    for i, (nx, ny, tau, fk, _, F0, a) in enumerate(spec):
        ref = orc.run(orc.init(*inits[i]), 100, tau, orc.Force(fk, F0, 4, a))
        err = rel_err(lat.get_populations_host(i), ref)
        assert err < FP32_TOL, (i, err)


@pytest.mark.parametrize("nx,ny", [(37, 23), (1, 1), (2, 5), (4, 1), (4, 3), (6, 130)])
def test_fp32_general_and_tiny_grids(P, orc, nx, ny):
    """Grids the vector kernel does not serve (nx % 4 != 0) and degenerate
    tiny grids (every neighbour is the cell itself)."""
    tau = 0.57
    m = P.Member(nx, ny, tau, 1.0, 1, 1, 1e-4, 1e-3)
    f0 = li.random_populations(nx, ny, seed=nx * 100 + ny, rel_noise=0.02)
    lat = P.Lattice([m], precision=32)
    lat.set_populations(0, f0)
    lat.step(100)
    ref = orc.run(f0, 100, tau, orc.Force(1, 1e-4, 1, 1e-3))
    assert rel_err(lat.get_populations_host(0), ref) < FP32_TOL


@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 3), (64, 64)])
def test_fp64_tiny_grids(P, orc, nx, ny):
    m = P.Member(nx, ny, 0.8, 1.0, 1, 1, 1e-4, 1e-3)
    f0 = li.random_populations(nx, ny, seed=7 + nx)
    lat = P.Lattice([m], precision=64)
    lat.set_populations(0, f0)
    lat.step(25)
    ref = orc.run(f0, 25, 0.8, orc.Force(1, 1e-4, 1, 1e-3))
    assert rel_err(lat.get_populations_host(0), ref) < FP64_TOL


def test_state_roundtrip(P):
    """set then get is the identity: bit-exact in FP64 (a permutation), within
    one FP32 rounding of the deviation in FP32."""
    nx, ny = 40, 12
    f0 = li.random_populations(nx, ny, seed=3)
    lat = P.Lattice([P.Member(nx, ny, 0.6)], precision=64)
    lat.set_populations(0, f0)
    assert np.array_equal(lat.get_populations_host(0), f0)
    import torch
    d = torch.from_numpy(f0).cuda()
    lat.set_populations(0, d)
    assert torch.equal(lat.get_populations(0), d)
    lat32 = P.Lattice([P.Member(nx, ny, 0.6)], precision=32)
    lat32.set_populations(0, f0)
    got = lat32.get_populations_host(0)
    assert np.max(np.abs(got - f0)) < 1e-8


def test_graph_replay_is_bitwise_identical(P):
    spec = _batch_members()
    members = [P.Member(nx, ny, tau, 1.0, fk, 4, F0, a) for (nx, ny, tau, fk, _, F0, a) in spec]
    outs = []
    for g in (0, 8):
        lat = P.Lattice(members, precision=32, graph_steps=g)
        for i, (nx, ny, *_r) in enumerate(spec):
            lat.init_fields(i, *_fields(nx, ny, 7 * i + 1))
        lat.step(37)
        outs.append([lat.get_populations_host(i) for i in range(len(spec))])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_decaying_ensemble_full_size_sampled(P, orc):
    """The 64-member 512^2 FP32 ensemble in the benchmark's launch shape:
    100 steps, two sampled members compared in full with the oracle."""
    wl = li.decaying_ensemble_workload()
    n, tau = wl["n"], wl["tau"]
    members = [P.Member(n, n, tau)] * wl["members"]
    lat = P.Lattice(members, precision=32, graph_steps=20, diag_every=wl["diag_every"])
    inits = {}
    for m in range(wl["members"]):
        r, u, v = li.random_phase(n, seed=wl["seed0"] + m, u_rms=wl["u_rms"])
        lat.init_fields(m, r, u, v)
        if m in (0, 45):
            inits[m] = (r, u, v)
    lat.step(100)
    for m, (r, u, v) in inits.items():
        ref = orc.run(orc.init(r, u, v), 100, tau)
        err = rel_err(lat.get_populations_host(m), ref)
        assert err < FP32_TOL, (m, err)
    for m in range(wl["members"]):
        assert lat.member_status(m) == 0


def test_divergence_flag(P):
    """A member seeded with NaN/negative density is flagged; the others not,
    and stepping the batch keeps working."""
    n = 32
    lat = P.Lattice([P.Member(n, n, 0.6)] * 3, precision=32)
    r, u, v = _fields(n, n, 5)
    for m in range(3):
        lat.init_fields(m, r, u, v)
    bad = r.copy()
    bad[3, 4] = np.nan
    lat.init_fields(1, bad, u, v)
    neg = r.copy()
    neg[0, 0] = -1.0
    lat.init_fields(2, neg, u, v)
    assert [lat.member_status(m) for m in range(3)] == [0, 1, 1]
    lat.step(3)
    assert lat.member_status(0) == 0 and lat.member_status(1) == 1


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("nx,ny", [(64, 64), (37, 23), (2, 5)])
def test_small_grid_persistent_run_is_bitwise_the_per_step_run(P, prec, storage, nx, ny):
    """A single small member on the general kernel without graph replay
    runs each lbm_step call in one cooperative launch (one launch counted);
    its states equal, bit for bit, those of the per-step launches (the same
    member in a two-member handle, the same handle stepped one step per
    call, and graph replay of per-step launches)."""
    if prec == 32 and nx % 4 == 0:
        pytest.skip("FP32 grids with nx % 4 == 0 take the vector kernel")
    m = P.Member(nx, ny, 0.57, 1.0, 1, 2, 2e-4, 1e-3)
    f0 = li.random_populations(nx, ny, seed=nx + ny, rel_noise=0.03)
    one = P.Lattice([m], precision=prec, storage=storage)
    two = P.Lattice([m, m], precision=prec, storage=storage)
    single = P.Lattice([m], precision=prec, storage=storage)
    graphs = P.Lattice([m], precision=prec, storage=storage, graph_steps=8)
    for lat in (one, two, single, graphs):
        for i in range(len(lat.members)):
            lat.set_populations(i, f0)
    c0 = one.launch_count
    one.step(101)
    assert one.launch_count - c0 == 1
    two.step(101)
    for _ in range(101):
        single.step(1)
    graphs.step(101)
    got = one.get_populations_host(0)
    assert np.array_equal(got, two.get_populations_host(0))
    assert np.array_equal(got, single.get_populations_host(0))
    assert np.array_equal(got, graphs.get_populations_host(0))
    assert not np.array_equal(got, f0)


def test_persistent_barrier_reports_a_withheld_arrival(P):
    """Failure detection of the grid barrier without any device fault: with
    every CTA arriving, 1000 barriers pass (no error); with one CTA that
    never arrives, the others give up after their bounded wait and the host
    reads the error word; the device stays usable."""
    import torch
    assert P.probe_grid_barrier(128, 1000) == 0
    assert P.probe_grid_barrier(64, 3, withhold=5) == 1
    assert P.probe_grid_barrier(128, 10) == 0
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum()) == 8.0
