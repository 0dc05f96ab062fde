"""The two closed forms the FP32 entropic collision uses (Sec. 1, ELBM),
against the oracle: the third-order series of the root alpha of
H(f + alpha Delta) = H(f) (below 1e-7 from the oracle's bisection root
while every relative departure |Delta / f| is below 0.02, error shrinking as
y^4, the first omitted order), and the product form of the equilibrium's
departure P_l - 1 (a few FP32 ulps from the oracle's entropic equilibrium,
relative accuracy kept at small u).  CPU only: both forms are restated here
from their derivations, the reference values come from the oracle."""
import numpy as np


def _series_root(f, d):
    y = d / f
    T = {k: float(np.sum(f * y ** k)) for k in range(2, 6)}
    u, q4, q5 = T[3] / T[2], T[4] / T[2], T[5] / T[2]
    c1 = u / 3.0
    c2 = 4.0 * u * u / 9.0 - 2.0 * q4 / 3.0
    c3 = 1.1 * q5 - 14.0 * u * q4 / 9.0 + 17.0 * u ** 3 / 27.0
    return 2.0 + c1 + c2 + c3


def _states(orc, rng, ymax, n):
    """Populations f (an entropic equilibrium of random moments) and a
    departure Delta with zero mass and momentum (the identity behind the
    entropy condition's form needs sum Delta = 0) scaled so that
    max |Delta / f| = ymax."""
    cx, cy, _ = orc.lattice()
    A = np.vstack([np.ones(9), cx, cy])
    out = []
    for _ in range(n):
        rho = 1.0 + 0.02 * rng.normal()
        f = orc.feq_entropic(rho, 0.05 * rng.normal(), 0.05 * rng.normal())
        d = rng.normal(size=9) * f
        d -= A.T @ np.linalg.solve(A @ A.T, A @ d)
        out.append((f, d * (ymax / np.max(np.abs(d / f)))))
    return out


def test_series_is_the_root_below_two_percent(orc):
    rng = np.random.default_rng(21)
    for ymax in (1e-4, 1e-3, 5e-3, 1e-2, 2e-2):
        worst = 0.0
        for f, d in _states(orc, rng, ymax, 30):
            a = orc.elbm_alpha(f, d)
            worst = max(worst, abs(_series_root(f, d) - a))
        assert worst < 1e-7, (ymax, worst)


def test_series_error_is_fourth_order(orc):
    """Halving the departures divides the error by about 2^4."""
    rng = np.random.default_rng(22)
    for f, d in _states(orc, rng, 0.04, 10):
        e1 = abs(_series_root(f, d) - orc.elbm_alpha(f, d))
        e2 = abs(_series_root(f, 0.5 * d) - orc.elbm_alpha(f, 0.5 * d))
        assert e1 > 1e-11
        assert 8.0 < e1 / e2 < 32.0, (e1, e2)


def _em_product_form_f32(ux, uy, cx, cy):
    """P_l(u) - 1 of the entropic equilibrium in the product form the FP32
    collision uses (each factor 1 + small, no logarithm), in FP32."""
    f32 = np.float32

    def axis(u):
        u = f32(u)
        s = np.sqrt(f32(1) + f32(3) * u * u)
        q = f32(f32(3) * u * u) / f32(f32(1) + s)
        n = f32(3) * u + q
        b = n / f32(f32(1) - u)
        bm = -(n / f32(f32(1) + f32(2) * u + q))
        return {0: -q, 1: f32(-q * b + (b - q)), -1: f32(-q * bm + (bm - q))}

    X, Y = axis(ux), axis(uy)
    return np.array([float(f32(X[cx[l]] * Y[cy[l]] + (X[cx[l]] + Y[cy[l]]))) for l in range(9)])


def test_equilibrium_product_form_matches_the_oracle(orc):
    """The FP32 departure P_l - 1 from the product form is within a few FP32
    ulps of the oracle's entropic equilibrium over |u| <= 0.2, and it keeps
    its accuracy at small u (no cancellation: relative, not absolute)."""
    cx, cy, t = orc.lattice()
    rng = np.random.default_rng(23)
    worst = 0.0
    for _ in range(500):
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        exact = orc.feq_entropic(1.0, ux, uy) / t - 1.0
        worst = max(worst, float(np.max(np.abs(_em_product_form_f32(ux, uy, cx, cy) - exact))))
    assert worst < 5e-7, worst
    for u in (1e-3, 1e-5):
        exact = orc.feq_entropic(1.0, u, -0.5 * u) / t - 1.0
        got = _em_product_form_f32(u, -0.5 * u, cx, cy)
        nz = np.abs(exact) > 0
        assert np.max(np.abs(got[nz] - exact[nz]) / np.abs(exact[nz])) < 1e-5
