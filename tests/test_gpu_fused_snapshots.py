"""The stream-collide step that also records the snapshot-ring entry of the
state it reads (FP32 vector kernel, members without the paper forcing or a
variable viscosity) against the separate snapshot kernel: the trajectories
and the three eq. (17) levels must be bit-identical, shown through the
populations and through bitwise-equal balance statistics and per-box terms
over two diagnostic periods (every ring slot rewritten), in both storages,
with and without CUDA-graph replay; and each fused snapshot saves a launch."""
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


def _members(P):
    return [P.Member(64, 48, 0.55), P.Member(64, 48, 0.6, 1.0, 1, 2, 2e-4, 1e-4),
            P.Member(128, 36, 0.52)]


def _init(lat, members):
    for m, mb in enumerate(members):
        r = 1.0 + li.smooth_fields(mb.nx, mb.ny, 300 + 3 * m, amp=0.01)
        u = li.smooth_fields(mb.nx, mb.ny, 301 + 3 * m, amp=0.03)
        v = li.smooth_fields(mb.nx, mb.ny, 302 + 3 * m, amp=0.03)
        lat.init_fields(m, r, u, v)


@pytest.mark.parametrize("storage,graph", [(1, 0), (2, 0), (1, 4), (2, 4)])
def test_fused_snapshots_bit_identical(P, storage, graph):
    D = 12
    members = _members(P)
    fused = P.Lattice(members, precision=32, diag_every=D, storage=storage, graph_steps=graph)
    plain = P.Lattice(members, precision=32, diag_every=0, storage=storage, graph_steps=graph)
    _init(fused, members)
    _init(plain, members)
    Ls = [2, 4, 8, 16]
    for period in range(2):
        c0f, c0p = fused.launch_count, plain.launch_count
        fused.step(D)
        plain.step(D - 2)
        for _ in range(2):
            plain.record_snapshot()
            plain.step(1)
        plain.record_snapshot()
        assert fused.time == plain.time == (period + 1) * D
        # three separate snapshot launches against one (the last level)
        assert (plain.launch_count - c0p) - (fused.launch_count - c0f) == 2
        for m in range(len(members)):
            assert np.array_equal(fused.get_populations_host(m), plain.get_populations_host(m))
            sf, bf = fused.subvolume_balance(m, Ls, per_box=True)
            sp, bp = plain.subvolume_balance(m, Ls, per_box=True)
            assert np.array_equal(sf, sp, equal_nan=True), (period, m)
            assert np.array_equal(bf.cpu().numpy(), bp.cpu().numpy(), equal_nan=True), (period, m)
    fused.close()
    plain.close()


def test_not_fused_with_paper_forcing(P):
    """A batch with a kind-2 member keeps the separate snapshot launches (its
    damping coefficients are recorded with each snapshot)."""
    D = 6
    members = [P.Member(64, 48, 0.55), P.Member(64, 48, 0.55, 1.0, 2, 0, 8e-4, 0.0, 0.0, 1e-5)]
    a = P.Lattice(members, precision=32, diag_every=D)
    b = P.Lattice(members, precision=32, diag_every=0)
    _init(a, members)
    _init(b, members)
    a.step(D)
    b.step(D - 2)
    for _ in range(2):
        b.record_snapshot()
        b.step(1)
    b.record_snapshot()
    for m in range(2):
        assert np.array_equal(a.get_populations_host(m), b.get_populations_host(m))
        assert np.array_equal(a.subvolume_balance(m, [4, 8]), b.subvolume_balance(m, [4, 8]),
                              equal_nan=True)
