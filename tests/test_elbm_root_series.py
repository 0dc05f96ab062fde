"""The third-order series of the entropic root that the FP32 collision uses
(Sec. 1, ELBM: alpha is the non-trivial root of H(f + alpha Delta) = H(f))
against the oracle's bisection root: below 1e-7 while every relative
departure |Delta / f| is below 0.02, and the error shrinks as y^4 (the first
omitted order).  CPU only: the series is restated here from its derivation,
the root comes from the oracle."""
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
