"""Pins of the three-dimensional (D3Q19, D3Q27) oracle against facts fixed by the
lattice, by the mathematics and by an independent symbolic evaluation of
the general index forms of eqs. (8)-(11), whose vortex-stretching term
RHS^{Omega,6} does not vanish in three dimensions."""
import numpy as np
import pytest

import lbm_inputs as li


def _smooth3(n, seed, amp):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    out = np.zeros((n, n, n))
    for _ in range(4):
        k = rng.integers(-2, 3, size=3)
        out += rng.normal() * np.cos(k[0] * X + k[1] * Y + k[2] * Z + rng.uniform(0, 2 * np.pi))
    return amp * out / np.max(np.abs(out))


@pytest.mark.parametrize("q", [19, 27])
def test_d3q_isotropy(orc, q):
    """sum t = 1, sum t c = 0, sum t c c = cs^2 I, fourth moments cs^4
    (delta delta + 2 perms), opposite pairs, no repeated velocity."""
    cx, cy, cz, t = orc.lattice3(q)
    assert len(t) == q and len({(a, b, c) for a, b, c in zip(cx, cy, cz)}) == q
    C = np.stack([cx, cy, cz], 1).astype(float)
    cs2 = 1.0 / 3.0
    assert abs(t.sum() - 1) < 1e-15
    assert np.max(np.abs(np.einsum("l,la->a", t, C))) < 1e-15
    np.testing.assert_allclose(np.einsum("l,la,lb->ab", t, C, C), cs2 * np.eye(3), atol=1e-15)
    M4 = np.einsum("l,la,lb,lc,ld->abcd", t, C, C, C, C)
    d = np.eye(3)
    want = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(M4, want, atol=1e-15)
    for l in range(q):
        assert sum(1 for m in range(q) if (C[m] == -C[l]).all()) == 1


def test_d3q27_is_the_tensor_product_lattice(orc):
    """D3Q27 = D1Q3 x D1Q3 x D1Q3: every velocity of {-1, 0, 1}^3 once, with
    weight w(c_x) w(c_y) w(c_z), w(0) = 2/3, w(+-1) = 1/6; its first 19
    velocities are the D3Q19 set in the same order."""
    cx, cy, cz, t = orc.lattice3(27)
    w1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}
    assert {(a, b, c) for a, b, c in zip(cx, cy, cz)} == {
        (a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)}
    for a, b, c, tl in zip(cx, cy, cz, t):
        assert abs(tl - w1[a] * w1[b] * w1[c]) < 1e-16
    c19 = orc.lattice3(19)
    for k in range(3):
        assert np.array_equal(c19[k], (cx, cy, cz)[k][:19])


@pytest.mark.parametrize("q", [19, 27])
def test_d3q_step_conserves_mass_and_adds_the_force(orc, q):
    n = 6
    rho, ux, uy, uz = 1 + _smooth3(n, 1, 0.01), _smooth3(n, 2, 0.03), _smooth3(n, 3, 0.03), \
        _smooth3(n, 4, 0.03)
    f = orc.init3(rho, ux, uy, uz, q=q)
    F0, kf, a = 3e-4, 1, 2e-3
    g = orc.run3(f, 1, 0.57, 1, F0, kf, a)
    cx, cy, cz, _ = orc.lattice3(q)
    m = orc.moments3(f)
    np.testing.assert_allclose(m["rho"], rho, rtol=1e-14)  # f_eq carries (rho, rho u)
    np.testing.assert_allclose(m["ux"], ux, atol=1e-15)
    m0 = orc.moments3(f, 1, F0, kf, a)
    assert abs(g.sum() - f.sum()) < 1e-12
    for C, Fk in ((cx, "Fx"), (cy, "Fy"), (cz, "Fz")):
        gain = np.einsum("l,lzyx->", C, g) - np.einsum("l,lzyx->", C, f)
        assert abs(gain - m0[Fk].sum()) < 1e-13


@pytest.mark.parametrize("q", [19, 27])
def test_d3q_shear_wave_decay_rate(orc, q):
    """u_x = U sin(2 pi z / N) decays as exp(-nu k^2 t), nu = (tau - 1/2)/3,
    to the lattice's O(k^2) corrections (within 1%)."""
    N, U, tau, steps = 32, 1e-4, 0.8, 300
    z = np.arange(N)
    shape = (N, 2, 2)
    ux = np.broadcast_to((U * np.sin(2 * np.pi * z / N))[:, None, None], shape).copy()
    f = orc.init3(np.ones(shape), ux, np.zeros(shape), np.zeros(shape), q=q)
    g = orc.run3(f, steps, tau)
    amp = orc.moments3(g)["ux"][:, 0, 0]
    fit = np.sum(amp * np.sin(2 * np.pi * z / N)) / np.sum(np.sin(2 * np.pi * z / N) ** 2)
    nu, k = (tau - 0.5) / 3.0, 2 * np.pi / N
    assert abs(fit / U / np.exp(-nu * k * k * steps) - 1.0) < 0.01


def test_d3_stencil_is_eq18_on_each_axis(orc):
    """Along every axis the derivative of sin(k x) has the modified
    wavenumber of eq. (18): (8/5) sin(k) - (2/5) sin(2k) + (8/105) sin(3k)
    - (1/140) sin(4k)."""
    n = 16
    k = 2 * np.pi * 3 / n
    kt = 1.6 * np.sin(k) - 0.4 * np.sin(2 * k) + 8 / 105 * np.sin(3 * k) - np.sin(4 * k) / 140
    i = np.arange(n)
    for axis in range(3):
        shape = [1, 1, 1]
        shape[2 - axis] = n
        A = np.broadcast_to(np.sin(k * i).reshape(shape), (n, n, n)).copy()
        want = np.broadcast_to((kt * np.cos(k * i)).reshape(shape), (n, n, n))
        np.testing.assert_allclose(orc.d3(A, axis), want, atol=1e-14)


def _symbolic_terms3(n, tau, t_n, wt):
    sp = pytest.importorskip("sympy")
    x, y, z, t = sp.symbols("x y z t", real=True)
    k = 2 * sp.pi / n
    R = sp.Rational
    rho = 1 + R(2, 100) * sp.cos(k * x + k * z + R(1, 3)) * sp.cos(wt * t)
    ux = R(2, 100) * sp.sin(k * y - R(1, 2) + wt * t) + R(1, 100) * sp.cos(k * z + k * y)
    uy = R(15, 1000) * sp.cos(k * x + R(7, 10)) * sp.cos(wt * t) - R(5, 1000) * sp.sin(k * z)
    uz = R(1, 100) * sp.sin(k * x + k * y + wt * t) + R(4, 1000) * sp.cos(k * y - k * z)
    Fx = R(3, 10000) * sp.sin(k * y)
    Fy = R(2, 10000) * sp.sin(k * z) * sp.cos(k * x)
    Fz = -R(1, 10000) * sp.cos(k * x - k * y)
    u, F, X = [ux, uy, uz], [Fx, Fy, Fz], [x, y, z]
    nu = R(1, 3) * (sp.nsimplify(tau) - R(1, 2))
    p = rho / 3
    d = lambda e, j: sp.diff(e, X[j])  # noqa: E731
    eps = sp.LeviCivita
    R3 = range(3)
    om = [sum(eps(i, j, kk) * d(u[kk], j) for j in R3 for kk in R3) for i in R3]
    E = rho * sum(ui * ui for ui in u) / 2
    Om = sum(o * o for o in om) / 2
    S = [[d(u[i], j) + d(u[j], i) for j in R3] for i in R3]
    H = [sum(d(nu * rho * S[i][j], j) for j in R3) / rho for i in R3]
    T = [
        sp.diff(E, t),
        -sum(d(E * u[j], j) for j in R3),
        -sum(u[i] * d(p, i) for i in R3),
        sum(u[i] * F[i] for i in R3),
        -sum(nu * rho * S[i][j] * d(u[i], j) for i in R3 for j in R3),
        sum(d(nu * rho * u[i] * S[i][j], j) for i in R3 for j in R3),
        sp.diff(Om, t),
        -sum(d(Om * u[j], j) for j in R3),
        -Om * sum(d(u[j], j) for j in R3),
        sum(om[i] * eps(i, j, kk) * d(F[kk] / rho, j) for i in R3 for j in R3 for kk in R3),
        sum(H[i] * eps(i, j, kk) * d(om[kk], j) for i in R3 for j in R3 for kk in R3),
        sum(d(eps(i, j, kk) * om[i] * H[kk], j) for i in R3 for j in R3 for kk in R3),
        sum(om[i] * om[j] * d(u[i], j) for i in R3 for j in R3),
    ]
    xs = np.arange(n, dtype=float)
    ZZ, YY, XX = np.meshgrid(xs, xs, xs, indexing="ij")

    def ev(e, tt):
        fn = sp.lambdify((x, y, z, t), e, "numpy")
        return np.broadcast_to(np.asarray(fn(XX, YY, ZZ, tt), dtype=float), XX.shape).copy()

    fields = {name: [ev(e, t_n - m) for m in range(3)]
              for name, e in (("rho", rho), ("ux", ux), ("uy", uy), ("uz", uz))}
    return [ev(e, t_n) for e in T], fields, [ev(e, t_n) for e in F]


def test_terms3_match_symbolic_continuum(orc):
    """Every discrete 3D term (eq. 18 stencils, eq. 17 in time) matches the
    exact continuum term of the general index forms on a smooth 3D field to
    the schemes' truncation error, vortex stretching included."""
    n, tau, wt, t_n = 48, 0.58, 2e-3, 10.0
    exact, fl, F = _symbolic_terms3(n, tau, t_n, wt)
    got = orc.terms3(tau, fl["rho"], fl["ux"], fl["uy"], fl["uz"], *F)
    for q in range(13):
        scale = max(np.max(np.abs(exact[q])), 1e-300)
        tol = 1e-5 if q in (0, 6) else 5e-7
        err = np.max(np.abs(got[q] - exact[q])) / scale
        assert err < tol, (orc.TERM_NAMES[q], err)
    assert np.max(np.abs(exact[12])) > 0.1 * np.max(np.abs(exact[8]))  # stretching is there


def test_terms3_divergence_terms_vanish_on_whole_domain(orc):
    n = 12
    rho3 = [1 + _smooth3(n, 10 + m, 0.01) for m in range(3)]
    u3 = [[_smooth3(n, 20 + 3 * m + c, 0.03) for m in range(3)] for c in range(3)]
    F = [_smooth3(n, 40 + c, 1e-4) for c in range(3)]
    T = orc.terms3(0.55, rho3, u3[0], u3[1], u3[2], *F)
    for q in (1, 5, 7, 11):
        assert abs(T[q].mean()) < 1e-14 * np.max(np.abs(T[q])), orc.TERM_NAMES[q]
    assert np.max(np.abs(T[12])) > 0


def test_box_mean3_brute_force(orc):
    rng = np.random.default_rng(9)
    A = rng.standard_normal((5, 4, 6))
    nz, ny, nx = A.shape
    for L in (1, 2, 4):
        for (x0, y0, z0) in [(0, 0, 0), (5, 3, 4), (2, 1, 3), (4, 0, 1)]:
            ref = np.roll(np.roll(np.roll(A, -z0, 0), -y0, 1), -x0, 2)[:L, :L, :L].mean()
            assert abs(orc.box_mean3(A, x0, y0, z0, L) - ref) < 1e-14


def test_balance_stats3_all_origins_mean_is_global(orc):
    n = 6
    T = np.stack([_smooth3(n, 50 + q, 1.0) + 0.1 * q for q in range(13)])
    st, pb = orc.balance_stats3(T, [1, 2, 6, 7], per_box=True)
    for iL in range(3):
        np.testing.assert_allclose(st[iL, 2:, 0], T.reshape(13, -1).mean(axis=1), atol=5e-14)
    assert np.all(np.isnan(st[3]))
    assert np.all(np.abs(st[2, 2:, 1]) < 1e-14)


@pytest.mark.parametrize("q", [19, 27])
def test_d3q_equilibrium_moments(orc, q):
    """The quadratic equilibrium reproduces rho, rho u and the Euler stress
    rho (cs^2 I + u u) exactly on lattices with fourth-order isotropy; at rest
    it is rho t_l."""
    cx, cy, cz, t = orc.lattice3(q)
    C = np.stack([cx, cy, cz], 1).astype(float)
    for rho, u in [(1.0, (0.0, 0.0, 0.0)), (1.04, (0.05, -0.03, 0.02)), (0.96, (-0.1, 0.07, 0.12))]:
        f = orc.feq3(rho, *u, q=q)
        u = np.array(u)
        assert abs(f.sum() - rho) < 1e-15
        np.testing.assert_allclose(C.T @ f, rho * u, rtol=0, atol=1e-16)
        np.testing.assert_allclose(np.einsum("la,lb,l->ab", C, C, f),
                                   rho * (np.eye(3) / 3.0 + np.outer(u, u)), rtol=0, atol=1e-15)
        if not u.any():
            np.testing.assert_allclose(f, rho * t, rtol=0, atol=1e-17)


@pytest.mark.parametrize("q", [19, 27])
def test_terms3_from_populations_uniform_states(orc, q):
    """Uniform states at n, n-1, n-2 with an energy quadratic in time: only
    LHS^E survives and equals the slope e1 (BDF2 is exact on quadratics),
    which fixes the order of the three levels."""
    n, tau, rho0 = 4, 0.6, 0.98
    e0, e1, e2 = 5e-4, -2e-5, 3e-6
    states = []
    for t in (0, -1, -2):
        sp = np.sqrt(2 * (e0 + e1 * t + e2 * t * t) / rho0)
        full = lambda v: np.full((n, n, n), v)  # noqa: E731
        states.append(orc.init3(full(rho0), full(0.48 * sp), full(-0.6 * sp), full(0.64 * sp), q=q))
    T = orc.terms3_from_populations(*states, tau)
    np.testing.assert_allclose(T[0], e1, rtol=1e-11, atol=0)
    assert np.max(np.abs(T[1:])) < 1e-17


def test_balancing_errors3_include_vortex_stretching(orc):
    """Eqs. (12), (13) in 3D on constant term fields, every box alike: an
    exact balance gives 0 only when the vortex-stretching term RHS^{O,6}
    takes part in the enstrophy sum; a known imbalance gives imbalance /
    max |RHS^i|; all-zero terms give 0 and a zero right-hand side +Inf."""
    n, L = 4, 2
    vals = np.zeros(13)
    vals[0] = 1.0
    vals[1:6] = [0.5, 0.25, -0.25, 0.75, -0.25]            # sums to LHS^E
    vals[6] = -2.0
    vals[7:13] = [-1.0, -0.5, -0.25, 0.0, 0.0, -0.25]       # RHS^{O,6} = -0.25 closes it
    T = np.broadcast_to(vals[:, None, None, None], (13, n, n, n)).copy()
    _, pb = orc.balance_stats3(T, [L], per_box=True)
    assert np.all(pb[0][:, 0] == 0.0) and np.all(pb[0][:, 1] == 0.0)
    T[12] += 0.5  # RHS^{O,6}: -0.25 -> 0.25; sum -1.5; max |RHS| = 1
    T[4] -= 0.3   # RHS^{E,4}: 0.75 -> 0.45; sum 0.7; max |RHS| = 0.5
    _, pb = orc.balance_stats3(T, [L], per_box=True)
    np.testing.assert_allclose(pb[0][:, 0], 0.3 / 0.5, rtol=1e-14)
    np.testing.assert_allclose(pb[0][:, 1], 0.5 / 1.0, rtol=1e-14)
    Z = np.zeros((13, n, n, n))
    _, pb = orc.balance_stats3(Z, [L], per_box=True)
    assert np.all(pb[0][:, :2] == 0.0)
    Z[6] = 1.0
    _, pb = orc.balance_stats3(Z, [L], per_box=True)
    assert np.all(pb[0][:, 1] == np.inf) and np.all(pb[0][:, 0] == 0.0)
