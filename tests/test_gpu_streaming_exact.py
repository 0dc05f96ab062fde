"""Streaming and indexing bit for bit: the left-hand side of eq. (1),
f_l(x + c_l, n + 1) = f*_l(x), on the GPU against the oracle's streaming.

The step kernels always collide before they stream, so streaming is isolated
by a collision that is exactly the identity in floating point: no force and
a relaxation time so large (tau = 2^80) that the BGK correction
(f - f^eq) / tau, below 1e-24 here, lies under half an ulp of every stored
value (each is checked to exceed 1e-12 in magnitude: the population f, or
the deviation f - t_l rho0 of FP32 storage), while the exact-difference term
is a sum of products with the zero velocity jump.  The step then moves every stored value
unchanged, so the state exported after n steps must equal, element for
element, the exported initial state streamed n times by the oracle
(``np.array_equal``).  Exporting maps a stored FP32 deviation g to
t_l rho0 + g, the same function of (l, g) before and after streaming, so the
comparison is exact for FP32 handles too.  Covered: FP64 and FP32 handles,
the double buffer and both phases of the in-place AA pattern, the vector
kernel (nx % 4 == 0) and the general kernel, ragged and tiny grids, a batch
of uneven members in one launch, graph replay, and one 512^2 member.
"""
import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu

TAU_IDENTITY = 2.0 ** 80


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1809_06735_gb300 as P
    P.load_library()
    return P


def _check_magnitudes(orc, f):
    """Every stored value far from zero (see the module docstring)."""
    _, _, t = orc.lattice()
    assert np.min(np.abs(f)) > 1e-12
    assert np.min(np.abs(f - t[:, None, None])) > 1e-12


def _streamed(orc, f, n):
    for _ in range(n):
        f = orc.stream(f)
    return f


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("nx,ny", [(37, 23), (1, 1), (4, 3), (64, 48)])
def test_streaming_is_the_oracle_permutation(P, orc, prec, storage, nx, ny):
    lat = P.Lattice([P.Member(nx, ny, TAU_IDENTITY)], precision=prec, storage=storage)
    lat.set_populations(0, li.random_populations(nx, ny, seed=nx * 31 + ny, rel_noise=0.05))
    f0 = lat.get_populations_host(0)
    _check_magnitudes(orc, f0)
    done = 0
    for n in (1, 2, 37):  # cumulative 1, 3, 40 steps: both AA phases
        lat.step(n)
        done += n
        assert np.array_equal(lat.get_populations_host(0), _streamed(orc, f0, done)), done


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("storage", [1, 2])
def test_streaming_of_an_uneven_batch_with_graph_replay(P, orc, prec, storage):
    sizes = [(37, 23), (1, 1), (4, 3), (136, 40), (8, 1), (2, 5)]
    lat = P.Lattice([P.Member(nx, ny, TAU_IDENTITY) for nx, ny in sizes], precision=prec,
                    storage=storage, graph_steps=4)
    f0 = []
    for i, (nx, ny) in enumerate(sizes):
        lat.set_populations(i, li.random_populations(nx, ny, seed=500 + i, rel_noise=0.05))
        f0.append(lat.get_populations_host(i))
        _check_magnitudes(orc, f0[-1])
    lat.step(37)
    for i in range(len(sizes)):
        assert np.array_equal(lat.get_populations_host(i), _streamed(orc, f0[i], 37)), sizes[i]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("storage", [1, 2])
def test_streaming_of_a_512_member(P, orc, prec, storage):
    n = 512
    lat = P.Lattice([P.Member(n, n, TAU_IDENTITY)], precision=prec, storage=storage)
    lat.set_populations(0, li.random_populations(n, n, seed=77, rel_noise=0.05))
    f0 = lat.get_populations_host(0)
    _check_magnitudes(orc, f0)
    done = 0
    for k in (1, 2, 37):
        lat.step(k)
        done += k
        assert np.array_equal(lat.get_populations_host(0), _streamed(orc, f0, done)), done
