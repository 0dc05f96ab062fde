"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds input generation only: initial density and velocity
fields, random populations for parity tests, forcing amplitudes of the
workloads and sub-volume origin lists.  It contains none of the lattice
Boltzmann arithmetic (no equilibrium, collision, streaming, stencil or box
average), so the CUDA library and the oracle stay independent of each other.

All arrays are numpy float64, shape ``[ny, nx]`` (x fast), unless stated.
Random numbers come from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import numpy as np

CS2 = 1.0 / 3.0  # lattice speed of sound squared (D2Q9), used by input recipes


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def taylor_green(nx: int, ny: int | None = None, u0: float = 0.01, rho0: float = 1.0,
                 pressure_consistent: bool = True):
    """Taylor-Green vortex u = (u0 sin x cos y, -u0 cos x sin y) with
    x = 2 pi i / nx, y = 2 pi j / ny.  With ``pressure_consistent`` the density
    carries the incompressible pressure p = -(rho0 u0^2 / 4)(cos 2x + cos 2y)
    as rho = rho0 + p / cs^2; otherwise rho = rho0."""
    ny = nx if ny is None else ny
    x = 2.0 * np.pi * np.arange(nx) / nx
    y = 2.0 * np.pi * np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)  # [ny, nx]
    ux = u0 * np.sin(X) * np.cos(Y)
    uy = -u0 * np.cos(X) * np.sin(Y)
    if pressure_consistent:
        p = -(rho0 * u0 * u0 / 4.0) * (np.cos(2 * X) + np.cos(2 * Y))
        rho = rho0 + p / CS2
    else:
        rho = np.full((ny, nx), rho0)
    return rho, ux, uy


def random_phase(n: int, seed: int, u_rms: float, k_peak: float = 8.0, rho0: float = 1.0):
    """Incompressible random-phase velocity on an n x n periodic grid.

    Streamfunction modes psi_hat(k) = A(k) exp(i theta), theta ~ U[0, 2 pi),
    with |psi_hat|^2 = E(k) / (pi k^3) and E(k) ~ k^4 exp(-2 (k / k_peak)^2),
    k = |k| in units of 2 pi / n; the k = 0 and Nyquist modes are zero.
    u = (d_y psi, -d_x psi) (spectral derivatives), scaled so that
    sqrt(<u_x^2 + u_y^2>) = u_rms.  The density is the zero-Mach one,
    rho = rho0 + p / cs^2 with the incompressible pressure of
    lap p = -rho0 d_i u_j d_j u_i.
    Returns (rho, ux, uy)."""
    rng = _rng(seed)
    kx = np.fft.rfftfreq(n, 1.0 / n)  # 0 .. n/2
    ky = np.fft.fftfreq(n, 1.0 / n)   # 0 .. n/2-1, -n/2 .. -1
    KX, KY = np.meshgrid(kx, ky)      # [n, n//2 + 1]
    k = np.sqrt(KX ** 2 + KY ** 2)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=k.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        E = k ** 4 * np.exp(-2.0 * (k / k_peak) ** 2)
        amp = np.sqrt(E / (np.pi * k ** 3))
    amp[k == 0] = 0.0
    if n % 2 == 0:
        amp[:, -1] = 0.0                 # kx = n/2
        amp[np.abs(KY) == n // 2] = 0.0  # ky = -n/2
    psi = np.fft.irfft2(amp * np.exp(1j * theta), s=(n, n))
    ph = np.fft.rfft2(psi)
    wx = 2.0 * np.pi * KX / n
    wy = 2.0 * np.pi * KY / n
    ux = np.fft.irfft2(1j * wy * ph, s=(n, n))
    uy = np.fft.irfft2(-1j * wx * ph, s=(n, n))
    s = u_rms / np.sqrt(np.mean(ux ** 2 + uy ** 2))
    ux *= s
    uy *= s
    # zero-Mach pressure: lap p = -rho0 (d_i u_j)(d_j u_i)
    def d(a, w):
        return np.fft.irfft2(1j * w * np.fft.rfft2(a), s=(n, n))
    dxu, dyu, dxv, dyv = d(ux, wx), d(ux, wy), d(uy, wx), d(uy, wy)
    src = -rho0 * (dxu * dxu + 2.0 * dyu * dxv + dyv * dyv)
    k2 = wx ** 2 + wy ** 2
    sh = np.fft.rfft2(src)
    with np.errstate(divide="ignore", invalid="ignore"):
        phat = np.where(k2 > 0, -sh / k2, 0.0)
    p = np.fft.irfft2(phat, s=(n, n))
    rho = rho0 + p / CS2
    return rho, ux, uy


def kolmogorov_F0(n: int, tau: float, kf: int, alpha: float, u_amp: float) -> float:
    """Amplitude F0 of the Kolmogorov force F0 (sin(2 pi kf y/n), sin(2 pi kf x/n))
    whose laminar response has velocity amplitude u_amp under viscosity
    nu = cs^2 (tau - 1/2) and linear drag alpha: F0 = u_amp (nu k^2 + alpha),
    k = 2 pi kf / n."""
    nu = CS2 * (tau - 0.5)
    k = 2.0 * np.pi * kf / n
    return u_amp * (nu * k * k + alpha)


# Typical magnitudes of near-rest D2Q9 populations, used only to shape random
# test inputs (any positive values are valid populations).
_REST_SCALE = np.array([0.44, 0.11, 0.11, 0.11, 0.11, 0.028, 0.028, 0.028, 0.028])


def random_populations(nx: int, ny: int, seed: int, rel_noise: float = 0.05) -> np.ndarray:
    """Random positive populations f[9, ny, nx] = scale_l (1 + rel_noise N(0,1))."""
    rng = _rng(seed)
    noise = rng.standard_normal((9, ny, nx))
    return _REST_SCALE[:, None, None] * (1.0 + rel_noise * noise)


def smooth_fields(nx: int, ny: int, seed: int, amp: float = 0.02, kmax: int = 6):
    """Smooth random periodic field (sum of random low-wavenumber Fourier modes),
    zero mean, max amplitude about ``amp``.  Used for diagnostic parity inputs."""
    rng = _rng(seed)
    x = 2.0 * np.pi * np.arange(nx) / nx
    y = 2.0 * np.pi * np.arange(ny) / ny
    # each mode c cos(a x + b y + ph) = c [cos(a x + ph) cos(b y) - sin(a x + ph) sin(b y)],
    # summed as two rank-one products (separable: fast on large grids)
    cols, rows = [], []
    for _ in range(12):
        a, b = rng.integers(0, kmax + 1, size=2)
        if a == 0 and b == 0:
            continue
        ph = rng.uniform(0, 2 * np.pi)
        c = rng.standard_normal()
        cols += [c * np.cos(b * y), -c * np.sin(b * y)]
        rows += [np.cos(a * x + ph), np.sin(a * x + ph)]
    out = np.stack(cols, axis=1) @ np.stack(rows, axis=0) if cols else np.zeros((ny, nx))
    m = np.max(np.abs(out))
    return amp * out / (m if m > 0 else 1.0)


def table1_count(L: int, n: int) -> int:
    """Number of random boxes per size (the paper's Table 1 for a 256^2 grid):
    1 box at L = n; 1000 for 100 <= L < 256; 5000 for 10 <= L < 100; 10000
    below.  For other n the thresholds scale with n / 256."""
    if L >= n:
        return 1
    s = n / 256.0
    if L >= 100 * s:
        return 1000
    if L >= 10 * s:
        return 5000
    return 10000


def table1_origins(n: int, L: int, seed: int, count: int | None = None) -> np.ndarray:
    """Random lower-left origins [count, 2] (x0, y0) of L x L boxes lying inside
    the n x n domain (uniform in [0, n - L]^2), count from ``table1_count``."""
    rng = _rng(seed)
    c = table1_count(L, n) if count is None else count
    return rng.integers(0, n - L + 1, size=(c, 2)).astype(np.int32)


# ---------------------------------------------------------------------------
# Workloads (grid, relaxation time, forcing, steps, box sizes).
# ---------------------------------------------------------------------------

def pow2_sizes(lo_exp: int, hi_exp: int, n: int):
    return [1 << e for e in range(lo_exp, hi_exp + 1) if (1 << e) <= n]


def taylor_green_workload():
    """Plain FP64 Taylor-Green: 64^2, tau 0.6, u0 0.01, 1000 steps, boxes
    L in {4, 8, 16, 32} every 100 steps."""
    return dict(name="taylor_green_64_fp64", n=64, tau=0.6, rho0=1.0, u0=0.01, steps=1000,
                diag_every=100, Ls=[4, 8, 16, 32], precision=64)


def decaying_ensemble_workload(members: int = 64, n: int = 512):
    """Decaying 2D turbulence ensemble: 64 members of 512^2, FP32 deviation
    populations, tau 0.52, random-phase init (seed 1000 + member, u_rms
    0.02), 20000 steps, boxes L = 2^1..2^8 every 200 steps."""
    return dict(name=f"decaying_ensemble_{members}x{n}sq_fp32", members=members, n=n,
                tau=0.52, rho0=1.0, u_rms=0.02, seed0=1000, steps=20000, diag_every=200,
                Ls=pow2_sizes(1, 8, n), precision=32)


def forced_sweep_workload():
    """Forced tau sweep: grids {256, 512, 1024}^2 x tau {0.505, 0.51, 0.52,
    0.55, 0.6}, Kolmogorov kf = 4 with F0 for u_rms 0.03, drag 1e-4."""
    members = []
    m = 0
    for n in (256, 512, 1024):
        for tau in (0.505, 0.51, 0.52, 0.55, 0.6):
            members.append(dict(n=n, tau=tau, kf=4, alpha=1e-4,
                                F0=kolmogorov_F0(n, tau, 4, 1e-4, 0.03), seed=2000 + m))
            m += 1
    return dict(name="forced_sweep_15_uneven_fp32", members=members, u_rms=0.03, steps=50000,
                diag_every=200, Ls=pow2_sizes(1, 9, 1024), precision=32)


def large_forced_workload(n: int = 8192):
    """Large single forced run: 8192^2, tau 0.51, kf 4, drag 1e-5."""
    return dict(name=f"large_forced_{n}sq_fp32", n=n, tau=0.51, kf=4, alpha=1e-5,
                F0=kolmogorov_F0(n, 0.51, 4, 1e-5, 0.03), u_rms=0.03, seed=0, steps=10000,
                diag_every=100, Ls=pow2_sizes(1, 12, n), precision=32)


def adjoint_workload(n: int = 256):
    """Differentiation: 256^2, tau 0.55, Kolmogorov kf 4 (drag 1e-4), objective
    the mean over n in [1000, 2000] of the L = 16 box (origin (0, 0)) average
    of the dissipation term."""
    tau = 0.55
    return dict(name=f"adjoint_{n}sq", n=n, tau=tau, kf=4, alpha=1e-4,
                F0=kolmogorov_F0(n, tau, 4, 1e-4, 0.03), u_rms=0.02, seed=0, n0=1000,
                n1=2000, L=16, box=(0, 0), checkpoint_every=100)
