"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names the passage it checks.  None of them re-derives the oracle's
own formula: they use identities, closed forms, special cases, brute force
and an independent symbolic derivation of the continuum balance equations.
"""
import json
import os

import numpy as np
import pytest

import lbm_inputs as li

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Lattice and equilibrium (eq. 2)
# --------------------------------------------------------------------------

def test_lattice_isotropy(orc):
    """D2Q9 weights: sum t = 1, sum t c = 0, sum t c c = cs^2 I,
    sum t c_a^4 = 3 cs^4, sum t cx^2 cy^2 = cs^4, opposite pairs exist."""
    cx, cy, t = orc.lattice()
    cs2 = 1.0 / 3.0
    assert abs(t.sum() - 1) < 1e-15
    assert abs((t * cx).sum()) < 1e-15 and abs((t * cy).sum()) < 1e-15
    assert abs((t * cx * cx).sum() - cs2) < 1e-15
    assert abs((t * cy * cy).sum() - cs2) < 1e-15
    assert abs((t * cx * cy).sum()) < 1e-15
    assert abs((t * cx ** 4).sum() - 3 * cs2 ** 2) < 1e-15
    assert abs((t * cx ** 2 * cy ** 2).sum() - cs2 ** 2) < 1e-15
    vel = set(zip(cx.tolist(), cy.tolist()))
    assert len(vel) == 9
    assert all((-a, -b) in vel for a, b in vel)


def test_equilibrium_moments(orc):
    """Eq. (2) reproduces rho, rho u and rho (cs^2 I + u u) exactly."""
    cx, cy, _ = orc.lattice()
    rng = np.random.default_rng(1)
    for _ in range(200):
        rho = rng.uniform(0.5, 2.0)
        ux, uy = rng.uniform(-0.2, 0.2, size=2)
        e = orc.feq(rho, ux, uy)
        tol = 4e-16 * rho * 10
        assert abs(e.sum() - rho) < tol
        assert abs((cx * e).sum() - rho * ux) < tol
        assert abs((cy * e).sum() - rho * uy) < tol
        assert abs((cx * cx * e).sum() - rho * (1 / 3 + ux * ux)) < tol
        assert abs((cx * cy * e).sum() - rho * ux * uy) < tol
        assert abs((cy * cy * e).sum() - rho * (1 / 3 + uy * uy)) < tol


# --------------------------------------------------------------------------
# Collision with exact-difference forcing (eq. 1, Sec. 3)
# --------------------------------------------------------------------------

def test_collision_mass_and_momentum(orc):
    """BGK conserves mass; the EDM term adds exactly F to the momentum, with
    F = F_ext - alpha j."""
    cx, cy, _ = orc.lattice()
    rng = np.random.default_rng(2)
    f = li.random_populations(1, 1, seed=3, rel_noise=0.2)[:, 0, 0]
    for tau in (0.505, 0.6, 1.0, 1.7):
        for _ in range(20):
            f = f * rng.uniform(0.8, 1.2, size=9)
            Fex, Fey = rng.uniform(-1e-3, 1e-3, size=2)
            alpha = rng.uniform(0, 1e-2)
            out = orc.collide_cell(f, tau, Fex, Fey, alpha)
            jx, jy = (cx * f).sum(), (cy * f).sum()
            assert abs(out.sum() - f.sum()) < 1e-15
            assert abs((cx * out).sum() - (jx + Fex - alpha * jx)) < 1e-15
            assert abs((cy * out).sum() - (jy + Fey - alpha * jy)) < 1e-15


def test_collision_relaxes_to_equilibrium(orc):
    """With tau = 1 and no force the post-collision state is f_eq itself;
    an equilibrium state is a fixed point of the collision for any tau."""
    cx, cy, _ = orc.lattice()
    f = li.random_populations(1, 1, seed=4, rel_noise=0.1)[:, 0, 0]
    rho = f.sum()
    ux, uy = (cx * f).sum() / rho, (cy * f).sum() / rho
    np.testing.assert_allclose(orc.collide_cell(f, 1.0, 0, 0, 0), orc.feq(rho, ux, uy),
                               rtol=2e-15, atol=0)
    e = orc.feq(1.1, 0.03, -0.02)
    for tau in (0.51, 0.8, 2.0):
        np.testing.assert_allclose(orc.collide_cell(e, tau, 0, 0, 0), e, rtol=2e-15, atol=0)


def test_edm_forcing_is_difference_of_equilibria(orc):
    """Sec. 3 EDM: starting from equilibrium at velocity u, a forced collision
    lands on the equilibrium at u + F/rho for any tau (special case where the
    BGK part vanishes)."""
    rho, ux, uy = 1.05, 0.02, -0.01
    Fx, Fy = 3e-4, -2e-4
    e = orc.feq(rho, ux, uy)
    for tau in (0.6, 1.3):
        out = orc.collide_cell(e, tau, Fx, Fy, 0.0)
        np.testing.assert_allclose(out, orc.feq(rho, ux + Fx / rho, uy + Fy / rho),
                                   rtol=2e-15, atol=0)


# --------------------------------------------------------------------------
# Streaming (eq. 1, left-hand side)
# --------------------------------------------------------------------------

def test_stream_moves_each_value_by_its_velocity(orc):
    cx, cy, _ = orc.lattice()
    nx, ny = 7, 5
    for l in range(9):
        for (x, y) in [(0, 0), (6, 4), (3, 2), (6, 0), (0, 4)]:
            f = np.zeros((9, ny, nx))
            f[l, y, x] = 1.0
            g = orc.stream(f)
            assert g.sum() == 1.0
            assert g[l, (y + cy[l]) % ny, (x + cx[l]) % nx] == 1.0


def test_stream_is_a_permutation_with_period_n(orc):
    """Streaming is a bijection; n steps on an n x n grid are the identity,
    bit for bit."""
    n = 6
    f = li.random_populations(n, n, seed=5)
    g = orc.stream(f)
    for l in range(9):
        assert np.array_equal(np.sort(g[l].ravel()), np.sort(f[l].ravel()))
    h = f
    for _ in range(n):
        h = orc.stream(h)
    assert np.array_equal(h, f)
    assert np.array_equal(g[0], f[0])


def test_step_conserves_mass_and_gains_total_force(orc):
    """One step of eq. (1): total mass exact; total momentum grows by sum F."""
    n = 12
    force = orc.Force(1, 2e-4, 2, 3e-3)
    f = li.random_populations(n, n, seed=6)
    m0 = orc.moments(f, force)
    g = orc.run(f, 1, 0.57, force)
    m1 = orc.moments(g, force)
    Fx = np.zeros((n, n))
    Fy = np.zeros((n, n))
    for y in range(n):
        for x in range(n):
            Fx[y, x], Fy[y, x] = orc.force_ext(n, n, force, x, y)
    Fx -= force.alpha * m0["jx"]
    Fy -= force.alpha * m0["jy"]
    assert abs(m1["rho"].sum() - m0["rho"].sum()) < 1e-12
    assert abs(m1["jx"].sum() - (m0["jx"].sum() + Fx.sum())) < 1e-13
    assert abs(m1["jy"].sum() - (m0["jy"].sum() + Fy.sum())) < 1e-13


def test_force_ext_is_kolmogorov(orc):
    """Force values at a few points against the closed form."""
    n, F0, kf = 16, 1e-3, 3
    f = orc.Force(1, F0, kf, 0.0)
    for (x, y) in [(0, 0), (1, 5), (15, 3), (7, 11)]:
        fx, fy = orc.force_ext(n, n, f, x, y)
        assert abs(fx - F0 * np.sin(2 * np.pi * kf * y / n)) < 1e-18
        assert abs(fy - F0 * np.sin(2 * np.pi * kf * x / n)) < 1e-18
    assert orc.force_ext(n, n, orc.NO_FORCE, 3, 3) == (0.0, 0.0)


# --------------------------------------------------------------------------
# Whole LBGK: viscosity of eq. (5)
# --------------------------------------------------------------------------

def _tg_rate(orc, n, tau=0.6, u0=1e-3):
    rho, ux, uy = li.taylor_green(n, u0=u0, pressure_consistent=True)
    f = orc.init(rho, ux, uy)
    nu = (tau - 0.5) / 3
    k = 2 * np.pi / n
    T = int(0.5 / (2 * nu * k * k))
    t1 = T // 4
    x = 2 * np.pi * np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    basis = np.sin(X) * np.cos(Y)
    f1 = orc.run(f, t1, tau)
    f2 = orc.run(f1, T - t1, tau)
    a1 = np.sum(orc.moments(f1)["ux"] * basis) / np.sum(basis ** 2)
    a2 = np.sum(orc.moments(f2)["ux"] * basis) / np.sum(basis ** 2)
    return -np.log(a2 / a1) / (T - t1), 2 * nu * k * k


def test_taylor_green_decay_rate(orc):
    """Taylor-Green amplitude decays as exp(-2 nu k^2 t), nu = cs^2 (tau - 1/2)
    (eq. 5), with a rate error that falls at second order in k."""
    r32, e32 = _tg_rate(orc, 32)
    r64, e64 = _tg_rate(orc, 64)
    err32, err64 = abs(r32 / e32 - 1), abs(r64 / e64 - 1)
    assert err32 < 5e-4 and err64 < 1e-4
    assert 3.0 < err32 / err64 < 5.5


def test_kolmogorov_laminar_amplitude_and_power_balance(orc):
    """Steady Kolmogorov flow: velocity amplitude F0 / (nu k^2 + alpha) and,
    globally, injected power <u.F> equals dissipation <eps> (eq. 8 at L = N:
    the flux terms vanish and the time derivative is zero)."""
    n, tau, kf, alpha, A = 32, 0.8, 1, 1e-3, 0.005
    F0 = li.kolmogorov_F0(n, tau, kf, alpha, A)
    force = orc.Force(1, F0, kf, alpha)
    z = np.zeros((n, n))
    f = orc.init(np.ones((n, n)), z, z)
    rate = (tau - 0.5) / 3 * (2 * np.pi * kf / n) ** 2 + alpha
    f = orc.run(f, int(12 / rate), tau, force)
    m = orc.moments(f, force)
    x = 2 * np.pi * kf * np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    ax = np.sum(m["ux"] * np.sin(Y)) / np.sum(np.sin(Y) ** 2)
    ay = np.sum(m["uy"] * np.sin(X)) / np.sum(np.sin(X) ** 2)
    assert abs(ax / A - 1) < 1e-2 and abs(ay / A - 1) < 1e-2
    g = orc.global_quantities(f, tau, force)
    assert abs(g[5] / g[6] - 1) < 1e-2


# --------------------------------------------------------------------------
# Derivatives, eqs. (17), (18)
# --------------------------------------------------------------------------

def test_ddx_ddy_modified_wavenumber(orc):
    """Eq. (18) on a periodic sine has the closed-form modified wavenumber
    (8/5) sin k - (2/5) sin 2k + (8/105) sin 3k - (1/140) sin 4k."""
    nx, ny = 40, 24
    xs = np.arange(nx)
    ys = np.arange(ny)
    X, Y = np.meshgrid(xs, ys)
    for m in range(1, nx // 2):
        k = 2 * np.pi * m / nx
        kt = 8 / 5 * np.sin(k) - 2 / 5 * np.sin(2 * k) + 8 / 105 * np.sin(3 * k) \
            - 1 / 140 * np.sin(4 * k)
        A = np.sin(k * X + 0.3)
        np.testing.assert_allclose(orc.ddx(A), kt * np.cos(k * X + 0.3), rtol=0, atol=5e-14)
        np.testing.assert_allclose(orc.ddy(A), 0 * A, rtol=0, atol=1e-15)
    for m in range(1, ny // 2):
        k = 2 * np.pi * m / ny
        kt = 8 / 5 * np.sin(k) - 2 / 5 * np.sin(2 * k) + 8 / 105 * np.sin(3 * k) \
            - 1 / 140 * np.sin(4 * k)
        A = np.cos(k * Y - 1.1)
        np.testing.assert_allclose(orc.ddy(A), -kt * np.sin(k * Y - 1.1), rtol=0, atol=5e-14)


def test_ddx_exact_on_polynomials_up_to_degree_8(orc):
    """Eq. (18) is an 8th-order centred difference: exact on polynomials of
    degree <= 8 away from the periodic seam, not exact at degree 9."""
    n = 40
    x = np.arange(n, dtype=float)
    inner = slice(4, n - 4)
    for deg in range(0, 10):
        p = ((x - 20.0) / 10.0) ** deg
        dp = deg * ((x - 20.0) / 10.0) ** max(deg - 1, 0) / 10.0
        A = np.tile(p, (3, 1))
        got = orc.ddx(A)[1, inner]
        err = np.max(np.abs(got - dp[inner]))
        if deg <= 8:
            assert err < 1e-13, (deg, err)
        else:
            assert err > 1e-9, (deg, err)
        got_y = orc.ddy(A.T.copy())[inner, 1]
        if deg <= 8:
            assert np.max(np.abs(got_y - dp[inner])) < 1e-13


def test_bdf2_exact_on_quadratics(orc):
    """Eq. (17) is exact for A(t) = a + b t + c t^2 (derivative b + 2 c t_n)."""
    rng = np.random.default_rng(7)
    a, b, c = rng.standard_normal((3, 50))
    tn = 17.0
    A = lambda t: a + b * t + c * t * t  # noqa: E731
    got = orc.bdf2(A(tn), A(tn - 1), A(tn - 2))
    np.testing.assert_allclose(got, b + 2 * c * tn, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Balance terms, eqs. (8)-(11): independent symbolic derivation
# --------------------------------------------------------------------------

def _symbolic_terms(n, tau, t_n, wt):
    """Continuum terms of eqs. (10)/(11) from the 3D index forms with the
    Levi-Civita symbol, differentiated symbolically, on the grid at t_n."""
    sp = pytest.importorskip("sympy")
    x, y, z, t = sp.symbols("x y z t", real=True)
    k = 2 * sp.pi / n
    rho = 1 + sp.Rational(3, 100) * sp.cos(k * x + 2 * k * y + sp.Rational(1, 3)) * sp.cos(wt * t)
    ux = sp.Rational(2, 100) * sp.sin(k * y - sp.Rational(1, 2) + wt * t) \
        + sp.Rational(1, 100) * sp.cos(2 * k * x + k * y)
    uy = sp.Rational(15, 1000) * sp.cos(k * x + sp.Rational(7, 10)) * sp.cos(wt * t) \
        - sp.Rational(5, 1000) * sp.sin(k * x - 2 * k * y)
    Fx = sp.Rational(3, 10000) * sp.sin(k * y) + sp.Rational(1, 10000) * sp.cos(k * x - k * y)
    Fy = -sp.Rational(2, 10000) * sp.sin(2 * k * x) * sp.cos(k * y)
    u = [ux, uy, sp.Integer(0)]
    F = [Fx, Fy, sp.Integer(0)]
    X = [x, y, z]
    nu = sp.Rational(1, 3) * (sp.nsimplify(tau) - sp.Rational(1, 2))
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
    XX, YY = np.meshgrid(xs, xs)
    args = (x, y, z, t)

    def ev(e, tt):
        fn = sp.lambdify(args, e, "numpy")
        v = fn(XX, YY, 0.0, tt)
        return np.broadcast_to(np.asarray(v, dtype=float), XX.shape).copy()

    fields = {name: [ev(e, t_n - m) for m in range(3)]
              for name, e in (("rho", rho), ("ux", ux), ("uy", uy))}
    Fxy = (ev(Fx, t_n), ev(Fy, t_n))
    return [ev(e, t_n) for e in T], fields, Fxy


def test_terms_match_symbolic_continuum(orc):
    """Every discrete term (eq. 18 stencils, eq. 17 in time) matches the exact
    continuum term of eqs. (10)/(11) on a smooth field to the schemes'
    truncation error; RHS^{Omega,6} vanishes in 2D."""
    n, tau, wt, t_n = 128, 0.58, 2e-3, 10.0
    exact, fl, (Fx, Fy) = _symbolic_terms(n, tau, t_n, wt)
    got = orc.terms(tau, fl["rho"], fl["ux"], fl["uy"], Fx, Fy)
    for q in range(13):
        scale = max(np.max(np.abs(exact[q])), 1e-300)
        if q == 12:
            assert np.max(np.abs(got[q])) == 0.0
            assert np.max(np.abs(exact[q])) < 1e-30
            continue
        # time derivatives carry the BDF2 error O(wt^2), space ones O(k^8)
        tol = 1e-5 if q in (0, 6) else 2e-8
        err = np.max(np.abs(got[q] - exact[q])) / scale
        assert err < tol, (orc.TERM_NAMES[q], err)


def test_divergence_terms_vanish_on_whole_domain(orc):
    """At L = N the flux terms RHS^{E,1}, RHS^{E,5}, RHS^{O,1}, RHS^{O,5}
    telescope to zero (centred differences on a periodic grid)."""
    n = 32
    fl = [li.smooth_fields(n, n, seed=s, amp=0.03) for s in range(10, 19)]
    rho3 = [1 + fl[0], 1 + fl[1], 1 + fl[2]]
    ux3, uy3 = fl[3:6], fl[6:9]
    Fx = li.smooth_fields(n, n, seed=30, amp=1e-4)
    Fy = li.smooth_fields(n, n, seed=31, amp=1e-4)
    T = orc.terms(0.55, rho3, ux3, uy3, Fx, Fy)
    for q in (1, 5, 7, 11):
        assert abs(T[q].mean()) < 1e-14 * np.max(np.abs(T[q])), orc.TERM_NAMES[q]
    assert np.all(T[12] == 0)


# --------------------------------------------------------------------------
# Sub-volume averages and balancing errors, eqs. (10)-(13), Table 1
# --------------------------------------------------------------------------

def test_box_mean_matches_brute_force_numpy(orc):
    """Box averages with periodic wrap against an independent numpy sum, every
    L and every origin on small grids (square and rectangular)."""
    rng = np.random.default_rng(8)
    for (ny, nx) in [(8, 8), (5, 7), (16, 12)]:
        A = rng.standard_normal((ny, nx))
        for L in range(1, min(nx, ny) + 1):
            for y0 in range(ny):
                for x0 in range(nx):
                    ref = np.roll(np.roll(A, -y0, axis=0), -x0, axis=1)[:L, :L].mean()
                    assert abs(orc.box_mean(A, x0, y0, L) - ref) < 1e-14


def test_all_origin_average_equals_global_mean(orc):
    """Averaging box means over all periodic origins gives the global mean for
    every L; at L = N every box is the whole domain (zero spread)."""
    n = 12
    T = np.stack([li.smooth_fields(n, n, seed=40 + q, amp=1.0) + 0.1 * q for q in range(13)])
    st = orc.balance_stats(T, [1, 3, 4, 12])
    for iL in range(4):
        np.testing.assert_allclose(st[iL, 2:, 0], T.reshape(13, -1).mean(axis=1),
                                   rtol=0, atol=5e-14)
    assert np.all(np.abs(st[3, 2:, 1]) < 1e-14)
    # L = 1 boxes are single cells: spread is the population std of the field
    np.testing.assert_allclose(st[0, 2:, 1], T.reshape(13, -1).std(axis=1), rtol=1e-12)


def test_balancing_error_special_cases(orc):
    """Eqs. (12), (13) on constant term fields: an exact balance gives 0, a
    known imbalance gives imbalance / max |RHS^i|."""
    n = 4
    vals = np.zeros(13)
    vals[0] = 1.0                               # LHS^E
    vals[1:6] = [0.5, 0.25, -0.25, 0.75, -0.25]  # sums to 1
    vals[6] = -2.0                              # LHS^O
    vals[7:13] = [-1.0, -0.5, -0.5, 0.0, 0.0, 0.0]
    T = np.broadcast_to(vals[:, None, None], (13, n, n)).copy()
    v = orc.box_values(T, 1, 2, 3)
    assert v[0] == 0.0 and v[1] == 0.0
    np.testing.assert_allclose(v[2:], vals, rtol=0, atol=1e-15)
    T[3] += 0.15  # RHS^{E,3}: -0.25 -> -0.10; sum 1.15; max |RHS| = 0.75
    T[7] -= 1.0   # RHS^{O,1}: -1 -> -2; sum -3; max |RHS| = 2
    v = orc.box_values(T, 0, 0, 2)
    assert abs(v[0] - 0.15 / 0.75) < 1e-15
    assert abs(v[1] - 1.0 / 2.0) < 1e-15
    Z = np.zeros((13, n, n))
    assert orc.box_values(Z, 0, 0, 2)[0] == 0.0
    Z[0] = 1.0
    assert orc.box_values(Z, 0, 0, 2)[0] == np.inf


def test_table1_box_counts_match_paper():
    """Number of sub-volumes per size, the paper's Table 1 (256^2 grid)."""
    with open(os.path.join(GOLDEN, "table1_box_counts.json")) as fh:
        g = json.load(fh)
    for row in g["rows"]:
        for L in row["L_examples"]:
            assert li.table1_count(L, g["grid"]) == row["count"], L
    o = li.table1_origins(256, 32, seed=1)
    assert o.shape == (5000, 2) and o.min() >= 0 and o.max() <= 256 - 32


def test_global_budget_of_decaying_run(orc):
    """Eq. (8) integrated over the periodic domain: the flux terms vanish, so
    d<E>/dt = -<eps> + <u.F> + <p div u>; the last (compressibility) term is
    small at low Mach, so the first two must close the budget to a few %."""
    n, tau = 32, 0.56
    rho, ux, uy = li.random_phase(n, seed=3, u_rms=0.02, k_peak=3.0)
    f = orc.init(rho, ux, uy)
    f = orc.run(f, 200, tau)  # let the initial acoustic transient relax
    g0 = orc.global_quantities(f, tau)
    f1 = orc.run(f, 1, tau)
    fm = orc.run(f, -0 + 0, tau)  # same state (no steps)
    assert np.array_equal(fm, f)
    f2 = orc.run(f1, 1, tau)
    e0 = g0[3]
    e2 = orc.global_quantities(f2, tau)[3]
    g1 = orc.global_quantities(f1, tau)
    dEdt = (e2 - e0) / 2.0
    assert abs(dEdt - (-g1[6] + g1[5])) < 0.05 * abs(g1[6])


def test_window_run_matches_full_run_inside_the_light_cone(orc):
    """A window of a larger periodic grid, forced at its global coordinates,
    reproduces the full run bit for bit on cells at least nsteps from its
    edges (used to check sampled cells of grids too large for the oracle)."""
    NX, NY, steps = 30, 26, 5
    force = orc.Force(1, 3e-4, 3, 2e-3)
    f0 = li.random_populations(NX, NY, seed=21)
    full = orc.run(f0, steps, 0.58, force)
    for (x0, y0, wx, wy) in [(3, 2, 16, 14), (25, 20, 12, 13), (0, 0, 11, 11)]:
        xs = (x0 + np.arange(wx)) % NX
        ys = (y0 + np.arange(wy)) % NY
        win = f0[:, ys][:, :, xs]
        got = orc.run_window(win, steps, 0.58, force, x0, y0, NX, NY)
        inner = (slice(None), slice(steps, wy - steps), slice(steps, wx - steps))
        want = full[:, ys][:, :, xs]
        assert np.array_equal(got[inner], want[inner])
        assert not np.array_equal(got, want)  # the edges are not valid


# --------------------------------------------------------------------------
# Sub-volume Mach number (eq. 20) and distributions over boxes (Sec. 4)
# --------------------------------------------------------------------------

def test_box_mach_uniform_flow(orc):
    """A uniform flow has Ma_V = |u| / c_s = |u| sqrt(3) in every box, every
    size, wrapping boxes included (eq. 20)."""
    ny, nx = 9, 13
    U, V = 0.021, -0.037
    ux, uy = np.full((ny, nx), U), np.full((ny, nx), V)
    want = np.hypot(U, V) * np.sqrt(3.0)
    for (x0, y0, L) in [(0, 0, 1), (12, 8, 5), (3, 2, 9), (7, 7, 4)]:
        assert abs(orc.box_mach(ux, uy, x0, y0, L) - want) < 1e-15


def test_box_mach_shear_rows_closed_form(orc):
    """u = (U sin(2 pi y / N), 0): the box mean of sin^2 over rows y0..y0+L-1
    is 1/2 - (1/2L) sum_j cos(a + j d), with the closed form of the sum
    sin(L d / 2) / sin(d / 2) cos(a + (L - 1) d / 2), a = 4 pi y0 / N,
    d = 4 pi / N (independent of the box's x extent)."""
    N, U = 24, 0.05
    y = np.arange(N)
    ux = np.tile((U * np.sin(2 * np.pi * y / N))[:, None], (1, N))
    uy = np.zeros((N, N))
    d = 4 * np.pi / N
    for (x0, y0, L) in [(0, 0, 5), (3, 20, 7), (11, 13, 10), (0, 5, 24)]:
        a = y0 * d
        s = np.sin(L * d / 2) / np.sin(d / 2) * np.cos(a + (L - 1) * d / 2)
        mean_sq = U * U * (0.5 - s / (2 * L))
        want = np.sqrt(mean_sq) * np.sqrt(3.0)
        assert abs(orc.box_mach(ux, uy, x0, y0, L) - want) < 1e-14 * want + 1e-16


def test_box_mach_taylor_green_whole_domain(orc):
    """Taylor-Green velocity U (sin x cos y, -cos x sin y) on a full period:
    <|u|^2> = U^2 / 2 exactly (discrete orthogonality), so the L = N box has
    Ma = U sqrt(3/2) at every origin."""
    N, U = 16, 0.03
    k = 2 * np.pi / N
    X, Y = np.meshgrid(np.arange(N), np.arange(N))
    ux = U * np.sin(k * X) * np.cos(k * Y)
    uy = -U * np.cos(k * X) * np.sin(k * Y)
    for (x0, y0) in [(0, 0), (5, 11), (15, 15)]:
        assert abs(orc.box_mach(ux, uy, x0, y0, N) - U * np.sqrt(1.5)) < 1e-15


def test_histogram_bin_rule(orc):
    """Bin of v = number of edges <= v: values equal to an edge go up, below
    the first edge to bin 0, +Inf to the last bin, NaN to none."""
    edges = [1e-6, 1e-4, 1e-2, 1.0]
    cases = {0.0: 0, 5e-7: 0, 1e-6: 1, 5e-5: 1, 1e-4: 2, 0.5: 3, 1.0: 4, 7.0: 4,
             float("inf"): 4, -1.0: 0}
    for v, b in cases.items():
        assert orc.hist_bin(v, edges) == b, v
    assert orc.hist_bin(float("nan"), edges) == -1


def test_distributions_count_every_box_once(orc):
    """The histograms hold every box exactly once, in the bin a brute-force
    count over the per-box balancing errors gives; Ma_V statistics equal the
    mean and population std of brute-force box values; L > N gives zero
    counts and NaN statistics."""
    rng = np.random.default_rng(3)
    ny, nx = 10, 12
    terms = rng.normal(size=(13, ny, nx))
    ux, uy = 0.05 * rng.normal(size=(ny, nx)), 0.05 * rng.normal(size=(ny, nx))
    Ls = [1, 3, 10, 11]
    de = np.geomspace(1e-3, 10.0, 9)
    me = np.linspace(0.0, 0.3, 7)
    origins = np.array([[0, 0], [11, 9], [5, 4], [2, 7], [5, 4]], dtype=np.int32)
    for org in (None, origins):
        hd, hm, ms = orc.distributions(terms, ux, uy, Ls, de, me, origins=org)
        _, pb = orc.balance_stats(terms, Ls, origins=org, per_box=True)
        boxes = [(b % nx, b // nx) for b in range(nx * ny)] if org is None else \
            [tuple(o) for o in org]
        for iL, L in enumerate(Ls):
            if L > min(nx, ny):
                assert hd[iL].sum() == 0 and hm[iL].sum() == 0 and np.all(np.isnan(ms[iL]))
                continue
            for q in range(2):
                want = np.zeros(len(de) + 1, dtype=np.int64)
                for b in range(len(boxes)):
                    want[sum(1 for e in de if e <= pb[iL, b, q])] += 1
                np.testing.assert_array_equal(hd[iL, q], want)
            mach = [np.sqrt(np.mean([ux[(y0 + j) % ny, (x0 + i) % nx] ** 2 +
                                     uy[(y0 + j) % ny, (x0 + i) % nx] ** 2
                                     for j in range(L) for i in range(L)]) * 3.0)
                    for (x0, y0) in boxes]
            want = np.zeros(len(me) + 1, dtype=np.int64)
            for m in mach:
                want[sum(1 for e in me if e <= m)] += 1
            np.testing.assert_array_equal(hm[iL], want)
            assert abs(ms[iL, 0] - np.mean(mach)) < 1e-14
            assert abs(ms[iL, 1] - np.std(mach)) < 1e-14


# --------------------------------------------------------------------------
# The paper's turbulence forcing: shell force (eqs. 14, 15), damping (eq. 16)
# --------------------------------------------------------------------------

def _half_shell(kmin2, kmax2):
    return [(kx, ky) for ky in range(0, 8) for kx in range(-7, 8)
            if kmin2 <= kx * kx + ky * ky <= kmax2 and (ky > 0 or kx > 0)]


def test_shell_force_is_spectral_curl_of_streamfunction(orc):
    """F^T = (d_y psi, -d_x psi) of the eq. (14) streamfunction: the oracle's
    analytic field equals the FFT derivative of psi sampled on the grid
    (non-square grid, non-zero phase), is divergence-free, and has Fourier
    support only on the shell 5 <= |k| <= 7."""
    nx, ny, F0, phi = 48, 40, 8e-4, 0.7
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    psi = np.zeros((ny, nx))
    for kx, ky in _half_shell(25, 49):
        psi += F0 * np.cos(2 * np.pi * (kx * X / nx + ky * Y / ny) + phi)
    KX = 2 * np.pi * np.fft.fftfreq(nx, 1.0 / nx)[None, :] / nx
    KY = 2 * np.pi * np.fft.fftfreq(ny, 1.0 / ny)[:, None] / ny
    ph = np.fft.fft2(psi)
    fx_want = np.real(np.fft.ifft2(1j * KY * ph))
    fy_want = np.real(np.fft.ifft2(-1j * KX * ph))
    f = orc.init(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
    Fx, Fy = orc.force_field(f, orc.Force(2, F0, 0, 0.0, phase=phi, FR0=0.0))
    scale = np.max(np.abs(fx_want))
    assert np.max(np.abs(Fx - fx_want)) < 1e-13 * scale
    assert np.max(np.abs(Fy - fy_want)) < 1e-13 * scale
    div = np.real(np.fft.ifft2(1j * KX * np.fft.fft2(Fx) + 1j * KY * np.fft.fft2(Fy)))
    assert np.max(np.abs(div)) < 1e-13 * scale
    kk = np.hypot(np.fft.fftfreq(nx, 1.0 / nx)[None, :], np.fft.fftfreq(ny, 1.0 / ny)[:, None])
    spec = np.abs(np.fft.fft2(Fx)) + np.abs(np.fft.fft2(Fy))
    assert np.max(spec[(kk < 5 - 1e-9) | (kk > 7 + 1e-9)]) < 1e-12 * np.max(spec)
    assert abs(Fx.mean()) < 1e-17 and abs(Fy.mean()) < 1e-17


def test_damping_removes_exactly_the_large_scale_modes(orc):
    """Eq. (16) on f = f_eq(1, u) (so j / rho = u exactly): the damping is
    -F^R_0 times the part of u on the modes 1 <= |k| <= 2 -- here the
    prescribed (1,0), (1,1), (0,2) components -- and ignores (2,1), (3,0)
    and the mean flow."""
    nx, ny, FR0 = 32, 24, 1e-5
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    ax, ay = 2 * np.pi * X / nx, 2 * np.pi * Y / ny
    inside_x = 0.01 * np.cos(ax) + 0.004 * np.sin(ax + ay)
    inside_y = -0.006 * np.cos(2 * ay + 0.3)
    outside_x = 0.003 * np.sin(2 * ax + ay) + 0.002 + 0.005 * np.cos(3 * ax)
    outside_y = 0.004 * np.cos(2 * ax + ay) - 0.001
    f = orc.init(np.ones((ny, nx)), inside_x + outside_x, inside_y + outside_y)
    Fx, Fy = orc.force_field(f, orc.Force(2, 0.0, 0, 0.0, phase=0.0, FR0=FR0))
    assert np.max(np.abs(Fx + FR0 * inside_x)) < 1e-18
    assert np.max(np.abs(Fy + FR0 * inside_y)) < 1e-18


def test_paper_forcing_step_conserves_mass_and_adds_the_total_force(orc):
    """One step with the paper's forcing and drag: mass is conserved and the
    momentum gained equals sum_x (F^T + F^R - alpha j) (EDM adds exactly F
    per cell); both forcing fields have zero mean, so the gain is the drag."""
    n = 24
    rho = 1.0 + li.smooth_fields(n, n, 3, amp=0.01)
    ux, uy = li.smooth_fields(n, n, 4, amp=0.03), li.smooth_fields(n, n, 5, amp=0.03)
    f = orc.init(rho, ux, uy)
    force = orc.Force(2, 8e-4, 0, 2e-3, phase=0.4, FR0=1e-3)
    g = orc.run(f, 1, 0.6, force)
    cx, cy, _ = orc.lattice()
    jx0 = np.einsum("l,lyx->yx", cx, f)
    jy0 = np.einsum("l,lyx->yx", cy, f)
    Fx, Fy = orc.force_field(f, force)
    assert abs(g.sum() - f.sum()) < 1e-12
    gain_x = np.einsum("l,lyx->", cx, g) - jx0.sum()
    gain_y = np.einsum("l,lyx->", cy, g) - jy0.sum()
    assert abs(gain_x - (Fx - 2e-3 * jx0).sum()) < 1e-13
    assert abs(gain_y - (Fy - 2e-3 * jy0).sum()) < 1e-13
    assert abs(gain_x + 2e-3 * jx0.sum()) < 1e-13


# --------------------------------------------------------------------------
# Variable-viscosity collisions (Sec. 1: Smagorinsky, eq. 7)
# --------------------------------------------------------------------------

def _pi_neq(orc, f9):
    cx, cy, _ = orc.lattice()
    rho = f9.sum()
    u = np.array([(cx * f9).sum(), (cy * f9).sum()]) / rho
    d = f9 - orc.feq(rho, u[0], u[1])
    C = np.stack([cx, cy], 1).astype(float)
    return rho, np.einsum("la,lb,l->ab", C, C, d)


def test_collision_models_keep_tau0_at_equilibrium(orc):
    """No non-equilibrium stress, no eddy viscosity: tau_eff = tau0."""
    f9 = orc.feq(1.02, 0.03, -0.05)
    for coll in (1, 2):
        m = orc.Force(0, collision=coll, Cs=0.1)
        assert orc.tau_eff(f9, 0.53, m) == 0.53


def test_smagorinsky_tau_solves_its_implicit_definition(orc):
    """nu_t = C sqrt(S:S) with S = -Pi^neq / (2 rho cs^2 tau_eff) evaluated at
    the returned tau_eff itself (numpy tensor algebra on the populations)."""
    rng = np.random.default_rng(7)
    for k in range(5):
        f9 = orc.feq(1.0 + 0.02 * rng.normal(), 0.05 * rng.normal(), 0.05 * rng.normal())
        f9 = f9 * (1.0 + 0.02 * rng.normal(size=9))
        tau0, C = 0.51 + 0.1 * k, 0.02 + 0.05 * k
        tau = orc.tau_eff(f9, tau0, orc.Force(0, collision=1, Cs=C))
        rho, Pi = _pi_neq(orc, f9)
        S = -Pi / (2.0 * rho / 3.0 * tau)
        assert tau > tau0
        assert abs((tau - tau0) / 3.0 - C * np.sqrt(np.sum(S * S))) < 1e-14


def test_eq7_viscosity_from_strain_traces(orc):
    """Eq. (7): nu_t = -(cs^2/3) tau0^2 Tr(S^3) / Tr(S^2), S from Pi^neq at
    tau0; traces by numpy matrix powers.  A traceless 2D strain has
    Tr(S^3) = 0 (eigenvalues +-s), so a pure shear keeps tau0."""
    rng = np.random.default_rng(8)
    for k in range(5):
        f9 = orc.feq(1.0 + 0.02 * rng.normal(), 0.05 * rng.normal(), 0.05 * rng.normal())
        f9 = f9 * (1.0 + 0.03 * rng.normal(size=9))
        tau0 = 0.52 + 0.05 * k
        tau = orc.tau_eff(f9, tau0, orc.Force(0, collision=2))
        rho, Pi = _pi_neq(orc, f9)
        S = -Pi / (2.0 * rho / 3.0 * tau0)
        nu_t = -(1.0 / 9.0) * tau0 ** 2 * np.trace(S @ S @ S) / np.trace(S @ S)
        assert abs((tau - tau0) / 3.0 - nu_t) < 1e-15 + 1e-12 * abs(nu_t)
    # pure shear: Pi^neq with only the xy component (add c_x c_y-odd mode)
    f9 = orc.feq(1.0, 0.0, 0.0)
    f9[[5, 7]] += 1e-4
    f9[[6, 8]] -= 1e-4
    assert orc.tau_eff(f9, 0.55, orc.Force(0, collision=2)) == pytest.approx(0.55, abs=1e-15)


def test_chapman_enskog_strain_from_nonequilibrium_stress(orc):
    """The relation the models use, Pi^neq = -2 rho cs^2 tau S: on a decaying
    BGK shear wave u_x = U sin(2 pi y / N) the measured Pi^neq_xy matches
    -rho cs^2 tau d_y u_x to about 1% (Chapman-Enskog, O(k^2) corrections)."""
    N, U, tau = 64, 0.01, 0.8
    y = np.arange(N)
    ux = np.tile((U * np.sin(2 * np.pi * y / N))[:, None], (1, 4))
    f = orc.run(orc.init(np.ones((N, 4)), ux, np.zeros((N, 4))), 200, tau)
    m = orc.moments(f)
    for yy in (5, 16, 40):
        _, Pi = _pi_neq(orc, f[:, yy, 0])
        k = 2 * np.pi / N
        amp = m["jx"][:, 0].max()  # current wave amplitude (rho ~ 1)
        dudy = amp * k * np.cos(k * yy)
        want = -(1.0 / 3.0) * tau * dudy
        assert abs(Pi[0, 1] - want) < 0.01 * abs(amp * k / 3.0 * tau)


def test_terms_take_a_local_viscosity(orc):
    """A constant viscosity field reproduces the tau form; RHS^{E,4} is
    pointwise proportional to the local viscosity."""
    n = 16
    rng = np.random.default_rng(4)
    rho3 = [1.0 + 0.01 * li.smooth_fields(n, n, 20 + k) for k in range(3)]
    ux3 = [li.smooth_fields(n, n, 30 + k) for k in range(3)]
    uy3 = [li.smooth_fields(n, n, 40 + k) for k in range(3)]
    Fx, Fy = np.zeros((n, n)), np.zeros((n, n))
    tau = 0.6
    T0 = orc.terms(tau, rho3, ux3, uy3, Fx, Fy)
    Tc = orc.terms(tau, rho3, ux3, uy3, Fx, Fy, nu=np.full((n, n), (tau - 0.5) / 3.0))
    np.testing.assert_array_equal(T0, Tc)
    nu = 0.01 + 0.02 * rng.random((n, n))
    Tv = orc.terms(tau, rho3, ux3, uy3, Fx, Fy, nu=nu)
    T1 = orc.terms(tau, rho3, ux3, uy3, Fx, Fy, nu=np.ones((n, n)))
    np.testing.assert_allclose(Tv[4], nu * T1[4], rtol=1e-14, atol=1e-30)
    np.testing.assert_array_equal(Tv[[0, 1, 2, 3, 6, 7, 8, 9]], T0[[0, 1, 2, 3, 6, 7, 8, 9]])


# --------------------------------------------------------------------------
# Entropic LBM (Sec. 1)
# --------------------------------------------------------------------------

def _H(f):
    _, _, t = __import__("oracle").lattice()
    return float(np.sum(f * np.log(f / t)))


def test_entropic_equilibrium_is_the_constrained_minimum_of_H(orc):
    """The closed form conserves rho and j exactly and equals a numerical
    minimisation of H = sum f ln(f/t) under those constraints (scipy)."""
    from scipy.optimize import minimize
    cx, cy, t = orc.lattice()
    for rho, ux, uy in [(1.0, 0.0, 0.0), (1.03, 0.05, -0.02), (0.97, -0.12, 0.08)]:
        feq = orc.feq_entropic(rho, ux, uy)
        assert abs(feq.sum() - rho) < 1e-15
        assert abs((cx * feq).sum() - rho * ux) < 1e-15
        assert abs((cy * feq).sum() - rho * uy) < 1e-15
        cons = [{"type": "eq", "fun": lambda f: f.sum() - rho},
                {"type": "eq", "fun": lambda f: (cx * f).sum() - rho * ux},
                {"type": "eq", "fun": lambda f: (cy * f).sum() - rho * uy}]
        x0 = t * rho * (1.0 + 0.1 * np.sin(np.arange(9)))
        res = minimize(lambda f: np.sum(f * np.log(f / t)), x0, constraints=cons,
                       bounds=[(1e-9, None)] * 9, method="SLSQP",
                       options={"ftol": 1e-15, "maxiter": 500})
        assert np.max(np.abs(res.x - feq)) < 1e-6


def test_elbm_alpha_satisfies_the_entropy_condition(orc):
    """H(f + alpha Delta) = H(f) by direct evaluation of H, alpha in (1,
    a_max); alpha -> 2 (BGK) as the state approaches equilibrium."""
    rng = np.random.default_rng(11)
    for k in range(6):
        feq = orc.feq_entropic(1.0 + 0.02 * rng.normal(), 0.05 * rng.normal(), 0.05 * rng.normal())
        f = feq * (1.0 + 0.05 * rng.normal(size=9))
        cx, cy, _ = orc.lattice()
        rho, jx, jy = f.sum(), (cx * f).sum(), (cy * f).sum()
        d = orc.feq_entropic(rho, jx / rho, jy / rho) - f
        a = orc.elbm_alpha(f, d)
        assert a > 1.0 and np.all(f + a * d > 0)
        assert abs(_H(f + a * d) - _H(f)) < 1e-13
    feq = orc.feq_entropic(1.0, 0.03, 0.01)
    for eps in (1e-3, 1e-5):
        f = feq * (1.0 + eps * np.cos(np.arange(9)))
        rho, jx, jy = f.sum(), (cx * f).sum(), (cy * f).sum()
        d = orc.feq_entropic(rho, jx / rho, jy / rho) - f
        assert abs(orc.elbm_alpha(f, d) - 2.0) < 50 * eps


def test_elbm_cell_conserves_mass_and_adds_the_force(orc):
    rng = np.random.default_rng(12)
    cx, cy, _ = orc.lattice()
    f = orc.feq_entropic(1.01, 0.04, -0.03) * (1.0 + 0.03 * rng.normal(size=9))
    Fex, Fey, drag = 2e-4, -1e-4, 1e-3
    out, a = orc.elbm_cell(f, 0.52, Fex, Fey, drag)
    jx, jy = (cx * f).sum(), (cy * f).sum()
    assert abs(out.sum() - f.sum()) < 1e-15
    assert abs((cx * out).sum() - jx - (Fex - drag * jx)) < 1e-15
    assert abs((cy * out).sum() - jy - (Fey - drag * jy)) < 1e-15
    assert 1.0 < a < 64.0


# --------------------------------------------------------------------------
# Objective of the adjoint: time-window mean of the box-averaged dissipation
# term RHS^{E,4} of the energy balance (eq. 8)
# --------------------------------------------------------------------------

def test_objective_closed_form_dissipation(orc):
    """n0 = n1 = 0: the box mean of -nu rho (2 (du/dx)^2 + (du/dy + dv/dx)^2
    + 2 (dv/dy)^2) (minus twice nu rho S:S, nu = (tau - 1/2)/3 by eq. 5) of an
    equilibrium state built from analytic fields whose four velocity
    derivatives and density all vary.  At the lowest mode of a 256^2 grid the
    eighth-order stencil of eq. (18) differs from d/dx by about 1e-13 of the
    derivative, so the exact derivatives fix the value (boxes with and without
    periodic wrap)."""
    n, tau = 256, 0.58
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / n
    y, x = np.mgrid[0:n, 0:n].astype(float)
    U, V, A, B = 0.02, -0.015, 0.011, 0.007
    rho = 1.0 + 0.05 * np.sin(k * x + 0.3) * np.cos(k * y - 0.2)
    ux = U * np.cos(k * y) + A * np.sin(k * x)
    uy = V * np.cos(k * x) + B * np.sin(k * y)
    dxu, dyu = A * k * np.cos(k * x), -U * k * np.sin(k * y)
    dxv, dyv = -V * k * np.sin(k * x), B * k * np.cos(k * y)
    eps = -nu * rho * (2 * dxu ** 2 + (dyu + dxv) ** 2 + 2 * dyv ** 2)
    f0 = orc.init(rho, ux, uy)
    for (bx, by, L) in [(0, 0, n), (10, 200, 16), (250, 3, 32), (100, 240, 64), (7, 9, 1)]:
        want = np.roll(np.roll(eps, -by, axis=0), -bx, axis=1)[:L, :L].mean()
        got = orc.objective(f0, tau, orc.NO_FORCE, 0, 0, bx, by, L)
        assert abs(got - want) <= 1e-10 * abs(want), (bx, by, L, got, want)


def test_objective_window_is_the_mean_of_its_steps(orc):
    """The objective over steps n0..n1 is the plain mean of the single-step
    objectives, and the single-step objective at step n is the n = 0
    objective of the state n steps later (forced, sheared flow)."""
    nx, ny, tau = 24, 20, 0.56
    force = orc.Force(1, 3e-4, 2, 2e-3)
    f0 = orc.init(1.0 + li.smooth_fields(nx, ny, 11, amp=0.01),
                  li.smooth_fields(nx, ny, 12, amp=0.03), li.smooth_fields(nx, ny, 13, amp=0.03))
    bx, by, L = 19, 15, 8  # wraps in both directions
    n0, n1 = 3, 7
    single = [orc.objective(f0, tau, force, n, n, bx, by, L) for n in range(n0, n1 + 1)]
    J = orc.objective(f0, tau, force, n0, n1, bx, by, L)
    assert abs(J - np.mean(single)) <= 1e-13 * abs(J)
    for n, Jn in zip(range(n0, n1 + 1), single):
        later = orc.run(f0, n, tau, force)
        assert abs(orc.objective(later, tau, force, 0, 0, bx, by, L) - Jn) <= 1e-14 * abs(Jn)
    # the window sees the dynamics: the single-step values are not all equal
    assert np.ptp(single) > 1e-6 * abs(J)


# --------------------------------------------------------------------------
# Grid-level assembly: collision of a whole grid, the local viscosity field,
# and the balance terms straight from three population snapshots
# --------------------------------------------------------------------------

def _perturbed_state(orc, nx, ny, seed):
    f = orc.init(1.0 + li.smooth_fields(nx, ny, seed, amp=0.02),
                 li.smooth_fields(nx, ny, seed + 1, amp=0.04),
                 li.smooth_fields(nx, ny, seed + 2, amp=0.04))
    rng = np.random.default_rng(seed)
    return f * (1.0 + 0.01 * rng.standard_normal(f.shape))  # non-equilibrium part


@pytest.mark.parametrize("force_args", [(0, 0.0, 0, 0.0), (0, 0.0, 0, 4e-3), (1, 3e-4, 2, 2e-3)])
def test_grid_collision_at_tau_one_is_the_shifted_equilibrium(orc, force_args):
    """Eq. (1) with the EDM term at tau = 1 forgets the incoming
    non-equilibrium part: the post-collision state is f^eq(rho, u + F/rho),
    u = j/rho, F = F_ext - alpha j (moments by numpy sums)."""
    nx, ny = 12, 10
    force = orc.Force(*force_args)
    f = _perturbed_state(orc, nx, ny, 50)
    cx, cy, _ = orc.lattice()
    rho = f.sum(axis=0)
    jx, jy = np.einsum("l,lyx->yx", cx, f), np.einsum("l,lyx->yx", cy, f)
    Fex, Fey = orc.force_field(f, force)
    Fx, Fy = Fex - force.alpha * jx, Fey - force.alpha * jy
    want = orc.init(rho, (jx + Fx) / rho, (jy + Fy) / rho)
    np.testing.assert_allclose(orc.collide(f, 1.0, force), want, rtol=0, atol=2e-16)


def test_grid_collision_is_affine_in_the_relaxation_rate_and_conserves(orc):
    """BGK moves f towards the equilibrium by the fraction 1/tau: the changes
    at two relaxation times, relative to tau = 1, scale as (1/tau - 1); every
    tau keeps the mass and adds the force F = F_ext - alpha j to the
    momentum."""
    nx, ny = 12, 10
    force = orc.Force(1, 3e-4, 2, 2e-3)
    f = _perturbed_state(orc, nx, ny, 60)
    cx, cy, _ = orc.lattice()
    p1 = orc.collide(f, 1.0, force)
    d = {tau: (orc.collide(f, tau, force) - p1) / (1.0 / tau - 1.0) for tau in (0.55, 0.8, 1.7)}
    np.testing.assert_allclose(d[0.55], d[1.7], rtol=0, atol=1e-14)
    np.testing.assert_allclose(d[0.8], d[1.7], rtol=0, atol=1e-14)
    jx, jy = np.einsum("l,lyx->yx", cx, f), np.einsum("l,lyx->yx", cy, f)
    Fex, Fey = orc.force_field(f, force)
    for tau in (0.55, 0.8, 1.7):
        p = orc.collide(f, tau, force)
        np.testing.assert_allclose(p.sum(axis=0), f.sum(axis=0), rtol=0, atol=1e-15)
        np.testing.assert_allclose(np.einsum("l,lyx->yx", cx, p), jx + Fex - force.alpha * jx,
                                   rtol=0, atol=1e-16)
        np.testing.assert_allclose(np.einsum("l,lyx->yx", cy, p), jy + Fey - force.alpha * jy,
                                   rtol=0, atol=1e-16)


def test_nu_field_is_the_local_viscosity_of_each_cell(orc):
    """BGK: (tau - 1/2)/3 everywhere (eq. 5); Smagorinsky and eq. (7): the
    viscosity of each cell's own relaxation time, and the Smagorinsky eddy
    viscosity never lowers it."""
    nx, ny, tau0 = 8, 6, 0.53
    f = _perturbed_state(orc, nx, ny, 70)
    assert np.all(orc.nu_field(f, tau0, orc.Force(0)) == (tau0 - 0.5) / 3.0)
    for coll, cs in ((1, 0.1), (2, 0.0)):
        m = orc.Force(0, collision=coll, Cs=cs)
        nu = orc.nu_field(f, tau0, m)
        for y in range(ny):
            for x in range(nx):
                assert nu[y, x] == pytest.approx((orc.tau_eff(f[:, y, x], tau0, m) - 0.5) / 3.0,
                                                 rel=0, abs=1e-17)
        if coll == 1:
            assert np.all(nu >= (tau0 - 0.5) / 3.0) and np.any(nu > (tau0 - 0.5) / 3.0)


def test_terms_from_populations_uniform_states(orc):
    """Uniform states at levels n, n-1, n-2 whose energy is quadratic in time
    (E = e0 + e1 t + e2 t^2 at t = 0, -1, -2): no gradient, no vorticity, so
    every term but LHS^E vanishes, and the BDF2 time derivative of eq. (17)
    gives LHS^E = e1 exactly (the level order matters: e2 != 0)."""
    nx, ny, tau, rho0 = 6, 5, 0.6, 1.07
    e0, e1, e2 = 4e-4, 3e-5, 2e-6
    states = []
    for t in (0, -1, -2):
        E = e0 + e1 * t + e2 * t * t
        sp = np.sqrt(2 * E / rho0)
        states.append(orc.init(np.full((ny, nx), rho0), np.full((ny, nx), 0.6 * sp),
                               np.full((ny, nx), -0.8 * sp)))
    T = orc.terms_from_populations(*states, tau)
    np.testing.assert_allclose(T[0], e1, rtol=1e-11, atol=0)
    assert np.max(np.abs(T[1:])) < 1e-17


# --------------------------------------------------------------------------
# Diagnostic velocity of the exact-difference forcing (Sec. 3)
# --------------------------------------------------------------------------

def test_diagnostic_velocity_is_the_mid_step_velocity_under_uniform_drag(orc):
    """A uniform state under drag alone stays uniform (streaming a uniform
    field changes nothing), so one step takes the momentum from j(n) to
    j(n+1) = j(n) + F = (1 - alpha) j(n) in every cell.  The physical velocity
    of the exact-difference method is the mean of the momenta before and after
    the force acts: u(n) = (j(n) + j(n+1)) / (2 rho).  At alpha = 0.1 a dropped
    or sign-flipped F/2 shift moves u by 5e-2 or 1e-1 of its value."""
    nx, ny, tau, alpha, rho0 = 5, 4, 0.7, 0.1, 1.04
    f = orc.init(np.full((ny, nx), rho0), np.full((ny, nx), 0.03), np.full((ny, nx), -0.02))
    force = orc.Force(0, alpha=alpha)
    m0 = orc.moments(f, force)
    m1 = orc.moments(orc.run(f, 1, tau, force), force)
    np.testing.assert_allclose(m1["rho"], m0["rho"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1["jx"], (1 - alpha) * m0["jx"], rtol=0, atol=1e-16)
    np.testing.assert_allclose(m1["jy"], (1 - alpha) * m0["jy"], rtol=0, atol=1e-16)
    for u, j in (("ux", "jx"), ("uy", "jy")):
        np.testing.assert_allclose(m0[u], (m0[j] + m1[j]) / (2 * m0["rho"]), rtol=0, atol=1e-16)


@pytest.mark.parametrize("force_args", [dict(kind=0, alpha=5e-3),
                                        dict(kind=1, F0=3e-4, kf=2, alpha=2e-3),
                                        dict(kind=2, F0=1e-4, phase=0.4, FR0=0.05, alpha=1e-3)])
def test_diagnostic_velocity_is_the_mean_of_pre_and_post_collision_velocities(orc, force_args):
    """Exact-difference forcing (Sec. 3) moves each cell's velocity from
    u = j/rho to u + F/rho inside the collision; its physical velocity is the
    midpoint.  So, cell by cell and for every force kind (the Kolmogorov force,
    the shell force with the eq. (16) damping of the same state, drag),
    u(n) = (j + j*) / (2 rho) with j* = sum_l c_l f*_l the momentum of the
    post-collision populations (collision alone; it keeps rho)."""
    nx, ny = 12, 10
    force = orc.Force(**force_args)
    f = _perturbed_state(orc, nx, ny, 60)
    cx, cy, _ = orc.lattice()
    post = orc.collide(f, 0.63, force)
    rho = f.sum(axis=0)
    m = orc.moments(f, force)
    for u, c in (("ux", cx), ("uy", cy)):
        mid = (np.einsum("l,lyx->yx", c, f) + np.einsum("l,lyx->yx", c, post)) / (2 * rho)
        np.testing.assert_allclose(m[u], mid, rtol=0, atol=1e-16)


# --------------------------------------------------------------------------
# Entropic LBM relaxation (Sec. 1): beta = 1/(2 tau0), tau_eff = 2 tau0/alpha
# --------------------------------------------------------------------------

def _shear_wave_rate(orc, model, N, U, tau0, t1=50, T=450):
    y = np.arange(N)
    basis = np.sin(2 * np.pi * y / N)[:, None]
    ux = np.tile(U * basis, (1, 4))
    f1 = orc.run(orc.init(np.ones((N, 4)), ux, np.zeros((N, 4))), t1, tau0, model)
    f2 = orc.run(f1, T - t1, tau0, model)
    a1 = np.sum(orc.moments(f1)["ux"] * basis) / np.sum(basis ** 2 * np.ones((1, 4)))
    a2 = np.sum(orc.moments(f2)["ux"] * basis) / np.sum(basis ** 2 * np.ones((1, 4)))
    return -np.log(a2 / a1) / (T - t1)


def test_elbm_shear_wave_decays_at_the_bgk_viscosity(orc):
    """Near equilibrium the entropic root tends to alpha = 2, so ELBM's
    relaxation alpha beta must reduce to BGK's 1/tau0 and its shear viscosity
    to nu = cs^2 (tau0 - 1/2) (eq. 5).  A small shear wave
    u_x = U sin(2 pi y / N) then decays at nu k^2 (k = 2 pi / N, up to the
    lattice's O(k^2) correction) and at the rate of the BGK wave with the same
    tau0.  A factor beta = 1/tau0 would relax at 2/tau0 (tau_eff = tau0/2,
    below the stability limit at tau0 = 0.8)."""
    N, U, tau0 = 64, 1e-3, 0.8
    k = 2 * np.pi / N
    nu = (tau0 - 0.5) / 3.0
    r_elbm = _shear_wave_rate(orc, orc.Force(0, collision=3), N, U, tau0)
    r_bgk = _shear_wave_rate(orc, orc.Force(0), N, U, tau0)
    assert abs(r_elbm / (nu * k * k) - 1) < 1e-3
    assert abs(r_elbm / r_bgk - 1) < 1e-5


def test_elbm_relaxes_each_cell_at_the_tau_of_its_viscosity(orc):
    """Without force the ELBM collision scales each cell's departure from its
    equilibrium by 1 - alpha beta; the relaxation time that the diagnostic's
    local viscosity reports (nu_field, eq. 5: tau_eff = 3 nu + 1/2) must be
    the one the collision applies: f*_l - f^eq_l = (1 - 1/tau_eff)(f_l - f^eq_l)
    for every population of every cell, on states far enough from equilibrium
    that alpha differs from 2 (tau_eff differs from tau0)."""
    nx, ny, tau0 = 6, 5, 0.53
    model = orc.Force(0, collision=3)
    cx, cy, _ = orc.lattice()
    f = orc.init(1.0 + li.smooth_fields(nx, ny, 80, amp=0.02),
                 li.smooth_fields(nx, ny, 81, amp=0.04), li.smooth_fields(nx, ny, 82, amp=0.04))
    f = f * (1.0 + 0.05 * np.random.default_rng(80).standard_normal(f.shape))
    post = orc.collide(f, tau0, model)
    te = 3.0 * orc.nu_field(f, tau0, model) + 0.5
    assert np.max(np.abs(te - tau0)) > 5e-3  # alpha is not the BGK value here
    for y in range(ny):
        for x in range(nx):
            a = f[:, y, x]
            rho = a.sum()
            feq = orc.feq_entropic(rho, (cx * a).sum() / rho, (cy * a).sum() / rho)
            np.testing.assert_allclose(post[:, y, x] - feq, (1 - 1 / te[y, x]) * (a - feq),
                                       rtol=0, atol=1e-15)
