"""GPU checks of the two population storages: the in-place AA pattern and
the double buffer give the same trajectories as the FP64 oracle (same bars
as the stream-collide parity tests), through both phases of AA, on the
vector kernel (nx % 4 == 0, warp-edge stores across tiles and the periodic
seam) and the general kernel (any nx, FP64 and FP32)."""
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


def rel_err(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


SPEC = [(136, 40, 0.52, 1, 1e-4, 1e-4), (256, 64, 0.6, 0, 0.0, 0.0), (4, 3, 0.55, 1, 2e-5, 0.0),
        (132, 17, 0.51, 0, 0.0, 1e-3), (8, 1, 0.7, 1, 1e-4, 0.0)]


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("steps", [1, 2, 37])
def test_fp32_vector_kernel_storages(P, orc, storage, steps):
    members = [P.Member(nx, ny, tau, 1.0, fk, 3, F0, a) for (nx, ny, tau, fk, F0, a) in SPEC]
    lat = P.Lattice(members, precision=32, storage=storage, graph_steps=4)
    assert lat.tuning()["storage"] == ("aa" if storage == 1 else "double_buffer")
    f0 = []
    for i, (nx, ny, *_r) in enumerate(SPEC):
        f = li.random_populations(nx, ny, seed=40 + i, rel_noise=0.03)
        lat.set_populations(i, f)
        f0.append(f)
    lat.step(steps)
    for i, (nx, ny, tau, fk, F0, a) in enumerate(SPEC):
        ref = orc.run(f0[i], steps, tau, orc.Force(fk, F0, 3, a))
        got = lat.get_populations_host(i)
        assert rel_err(got, ref) < 2e-6, (storage, steps, i)


@pytest.mark.parametrize("prec,tol", [(64, 1e-12), (32, 2e-6)])
@pytest.mark.parametrize("nx,ny", [(37, 23), (1, 1), (2, 5), (64, 48)])
def test_general_kernel_aa(P, orc, prec, tol, nx, ny):
    m = P.Member(nx, ny, 0.58, 1.0, 1, 2, 2e-4, 1e-3)
    f0 = li.random_populations(nx, ny, seed=nx + 7 * ny, rel_noise=0.03)
    lat = P.Lattice([m], precision=prec, storage=1)
    lat.set_populations(0, f0)
    for k in (1, 4, 11):  # odd, even and odd phases
        lat.step(1 if k == 1 else (3 if k == 4 else 7))
        ref = orc.run(f0, k, 0.58, orc.Force(1, 2e-4, 2, 1e-3))
        assert rel_err(lat.get_populations_host(0), ref) < tol, k


def test_aa_odd_phase_roundtrip_and_diagnostic(P, orc):
    """set/get at an odd AA phase is the identity; snapshots and the balance
    of an AA run equal those of a double-buffer run to FP64 rounding."""
    n = 64
    f0 = li.random_populations(n, n, seed=5, rel_noise=0.01)
    lat = P.Lattice([P.Member(n, n, 0.6)], precision=64, storage=1, diag_every=21)
    lat.set_populations(0, f0)
    lat.step(1)
    g = lat.get_populations_host(0)
    lat.set_populations(0, g)
    assert np.array_equal(lat.get_populations_host(0), g)
    lat.step(20)
    st_aa = lat.subvolume_balance(0, [4, 16])
    ref = P.Lattice([P.Member(n, n, 0.6)], precision=64, storage=2, diag_every=21)
    ref.set_populations(0, f0)
    ref.step(21)
    st_db = ref.subvolume_balance(0, [4, 16])
    np.testing.assert_allclose(st_aa, st_db, rtol=1e-12, atol=1e-18)


def test_autotuned_storage_large_ensemble(P, orc):
    """An ensemble above the tuning threshold picks its storage and shape at
    create time; the chosen configuration still matches the oracle."""
    n, members = 512, 8
    lat = P.Lattice([P.Member(n, n, 0.52)] * members, precision=32, storage=0, graph_steps=10)
    tune = lat.tuning()
    assert tune["storage"] in ("aa", "double_buffer") and tune["tuned_step_ms"] > 0
    fields = li.random_phase(n, seed=3, u_rms=0.02)
    for m in range(members):
        lat.init_fields(m, *fields)
    lat.step(21)
    ref = orc.run(orc.init(*fields), 21, 0.52)
    assert rel_err(lat.get_populations_host(members - 1), ref) < 2e-6
