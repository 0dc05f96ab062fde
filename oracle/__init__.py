"""Python access to the FP64 CPU oracle (``lbm_oracle.c``, and
``lbm_oracle3d.c`` for the three-dimensional D3Q19 extension).

TEST INFRASTRUCTURE ONLY: the oracle is a plain, slow restatement of the
D2Q9 LBGK method (eqs. (1), (2) with exact-difference forcing) and of the
sub-volume energy/enstrophy balance diagnostic (eqs. (8)-(13), (17), (18)) of
Tauzin et al. (2018).  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library and never imports the product package.

Arrays are numpy float64, C-contiguous: populations ``f[9, ny, nx]`` and
fields ``A[ny, nx]`` (x is the fast index).  Term-field order:
``0 LHS^E, 1..5 RHS^{E,1..5}, 6 LHS^Omega, 7..12 RHS^{Omega,1..6}``.
Box statistics order: ``[delta^E, delta^Omega, <13 terms>]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SRC3 = os.path.join(_HERE, "lbm_oracle3d.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

NT = 13  # term fields
NQ = 15  # box quantities (2 balancing errors + 13 terms)
TERM_NAMES = ["LHS_E", "RHS_E1", "RHS_E2", "RHS_E3", "RHS_E4", "RHS_E5",
              "LHS_Z", "RHS_Z1", "RHS_Z2", "RHS_Z3", "RHS_Z4", "RHS_Z5", "RHS_Z6"]
QUANTITY_NAMES = ["delta_E", "delta_Z"] + TERM_NAMES


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3))):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99",
                               "-ffp-contract=off", "-o", tmp, _SRC, _SRC3, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            lib.orc_feq.argtypes = [D, D, D, P]
            lib.orc_force_ext.argtypes = [I, I, P, I, I, P, P]
            lib.orc_force_field.argtypes = [I, I, P, P, P, P]
            lib.orc_collide_cell.argtypes = [P, D, D, D, D, P]
            lib.orc_collide.argtypes = [I, I, D, P, P, P]
            lib.orc_collide.restype = I
            lib.orc_stream.argtypes = [I, I, P, P]
            lib.orc_run.argtypes = [I, I, D, P, P, I]
            lib.orc_run.restype = I
            lib.orc_run_window.argtypes = [I, I, D, P, P, I, I, I, I, I]
            lib.orc_run_window.restype = I
            lib.orc_init.argtypes = [I, I, P, P, P, P]
            lib.orc_moments.argtypes = [I, I, P, P, P, P, P, P, P]
            lib.orc_moments.restype = I
            lib.orc_ddx.argtypes = [I, I, P, P]
            lib.orc_ddy.argtypes = [I, I, P, P]
            lib.orc_bdf2.argtypes = [ctypes.c_size_t, P, P, P, P]
            lib.orc_terms.argtypes = [I, I, D, P, P, P, P, P, P, P]
            lib.orc_tau_eff.argtypes = [P, D, P]
            lib.orc_tau_eff.restype = D
            lib.orc_nu_field.argtypes = [I, I, D, P, P, P]
            lib.orc_feq_entropic.argtypes = [D, D, D, P]
            lib.orc_elbm_alpha.argtypes = [P, P]
            lib.orc_elbm_alpha.restype = D
            lib.orc_elbm_cell.argtypes = [P, D, D, D, D, P]
            lib.orc_elbm_cell.restype = D
            lib.orc_terms.restype = I
            lib.orc_box_mean.argtypes = [I, I, P, I, I, I]
            lib.orc_box_mean.restype = D
            lib.orc_box_values.argtypes = [I, I, P, I, I, I, P]
            lib.orc_balance_stats.argtypes = [I, I, P, P, I, P, I, P, P]
            lib.orc_balance_stats.restype = I
            lib.orc_terms_from_populations.argtypes = [I, I, D, P, P, P, P, P]
            lib.orc_terms_from_populations.restype = I
            lib.orc_global.argtypes = [I, I, D, P, P, P]
            lib.orc_global.restype = I
            lib.orc_objective.argtypes = [I, I, D, P, P, I, I, I, I, I, P]
            lib.orc_objective.restype = I
            lib.orc_lattice.argtypes = [P, P, P]
            lib.orc3_lattice.argtypes = [I, P, P, P, P]
            lib.orc3_lattice.restype = I
            lib.orc3_feq.argtypes = [I, D, D, D, D, P]
            lib.orc3_run.argtypes = [I, I, I, I, D, I, D, I, D, P, I]
            lib.orc3_run.restype = I
            lib.orc3_init.argtypes = [I, I, I, I, P, P, P, P, P]
            lib.orc3_moments.argtypes = [I, I, I, I, I, D, I, D, P, P, P, P, P, P, P, P]
            lib.orc3_d.argtypes = [I, I, I, I, P, P]
            lib.orc3_terms.argtypes = [I, I, I, D, P, P, P, P, P, P, P, P]
            lib.orc3_terms.restype = I
            lib.orc3_terms_from_populations.argtypes = [I, I, I, I, D, I, D, I, D, P, P, P, P]
            lib.orc3_terms_from_populations.restype = I
            lib.orc3_box_mean.argtypes = [I, I, I, P, I, I, I, I]
            lib.orc3_box_mean.restype = D
            lib.orc3_balance_stats.argtypes = [I, I, I, P, P, I, P, I, P, P]
            lib.orc3_balance_stats.restype = I
            lib.orc_box_mach.argtypes = [I, I, P, P, I, I, I]
            lib.orc_box_mach.restype = D
            lib.orc_bin.argtypes = [D, P, I]
            lib.orc_bin.restype = I
            lib.orc_distributions.argtypes = [I, I, P, P, P, P, I, P, I, P, I, P, I, P, P, P]
            lib.orc_distributions.restype = I
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class _ForceC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("F0", ctypes.c_double), ("kf", ctypes.c_int),
                ("alpha", ctypes.c_double), ("phase", ctypes.c_double), ("FR0", ctypes.c_double),
                ("collision", ctypes.c_int), ("Cs", ctypes.c_double)]


class Force:
    """Model of one member.  Forcing: kind 1 = Kolmogorov amplitude F0 at
    wavenumber kf (in units of 2 pi / N); kind 2 = the paper's shell force of
    eqs. (14), (15) (F^T_0 = F0, phase) plus the damping of eq. (16)
    (F^R_0 = FR0); in every case drag alpha on the bare momentum.  Collision:
    0 BGK, 1 Smagorinsky (constant Cs), 2 the turbulent viscosity of eq. (7),
    3 the entropic LBM."""

    def __init__(self, kind: int = 0, F0: float = 0.0, kf: int = 0, alpha: float = 0.0,
                 phase: float = 0.0, FR0: float = 0.0, collision: int = 0, Cs: float = 0.0):
        self.kind, self.F0, self.kf, self.alpha = int(kind), float(F0), int(kf), float(alpha)
        self.phase, self.FR0 = float(phase), float(FR0)
        self.collision, self.Cs = int(collision), float(Cs)
        self._c = _ForceC(self.kind, self.F0, self.kf, self.alpha, self.phase, self.FR0,
                          self.collision, self.Cs)

    def ptr(self):
        return ctypes.byref(self._c)


NO_FORCE = Force()


def lattice():
    lib = _load()
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    t = np.zeros(9)
    lib.orc_lattice(_p(cx), _p(cy), _p(t))
    return cx, cy, t


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_feq(rho, ux, uy, _p(out))
    return out


def feq_entropic(rho, ux, uy):
    """The D2Q9 entropic equilibrium (minimiser of H = sum f ln(f/t))."""
    out = np.zeros(9)
    _load().orc_feq_entropic(float(rho), float(ux), float(uy), _p(out))
    return out


def elbm_alpha(f9, delta9):
    """Non-trivial root alpha of H(f + alpha Delta) = H(f)."""
    f9, delta9 = _f64(f9), _f64(delta9)
    return _load().orc_elbm_alpha(_p(f9), _p(delta9))


def elbm_cell(f9, tau0, Fex=0.0, Fey=0.0, alpha_drag=0.0):
    """(post-collision populations, alpha) of one ELBM collision."""
    f9 = _f64(f9)
    out = np.zeros(9)
    a = _load().orc_elbm_cell(_p(f9), float(tau0), float(Fex), float(Fey), float(alpha_drag),
                              _p(out))
    return out, a


def tau_eff(f9, tau0, model: Force):
    """Local relaxation time of one cell's populations for the collision model."""
    f9 = _f64(f9)
    return _load().orc_tau_eff(_p(f9), float(tau0), model.ptr())


def nu_field(f, tau0, model: Force):
    """Local viscosity (tau_eff - 1/2)/3 of every cell of the state f."""
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.empty((ny, nx))
    _load().orc_nu_field(nx, ny, float(tau0), model.ptr(), _p(f), _p(out))
    return out


def force_field(f, force: Force):
    """External force (Fx, Fy) [ny, nx] of every cell for the state f, drag
    excluded: the static force plus, for kind 2, the damping of eq. (16)."""
    f = _f64(f)
    _, ny, nx = f.shape
    Fx, Fy = np.empty((ny, nx)), np.empty((ny, nx))
    _load().orc_force_field(nx, ny, force.ptr(), _p(f), _p(Fx), _p(Fy))
    return Fx, Fy


def force_ext(nx, ny, force: Force, x, y):
    fx, fy = ctypes.c_double(), ctypes.c_double()
    _load().orc_force_ext(nx, ny, force.ptr(), x, y, ctypes.byref(fx), ctypes.byref(fy))
    return fx.value, fy.value


def collide_cell(f9, tau, Fex, Fey, alpha):
    f9 = _f64(f9)
    out = np.zeros(9)
    _load().orc_collide_cell(_p(f9), tau, Fex, Fey, alpha, _p(out))
    return out


def collide(f, tau, force: Force = NO_FORCE):
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.empty_like(f)
    if _load().orc_collide(nx, ny, tau, force.ptr(), _p(f), _p(out)) != 0:
        raise MemoryError("oracle collide failed")
    return out


def stream(f):
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.empty_like(f)
    _load().orc_stream(nx, ny, _p(f), _p(out))
    return out


def init(rho, ux, uy):
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    ny, nx = rho.shape
    f = np.empty((9, ny, nx))
    _load().orc_init(nx, ny, _p(rho), _p(ux), _p(uy), _p(f))
    return f


def run(f, nsteps, tau, force: Force = NO_FORCE):
    """Return f after nsteps steps of eq. (1) (input not modified)."""
    f = _f64(f).copy()
    _, ny, nx = f.shape
    rc = _load().orc_run(nx, ny, tau, force.ptr(), _p(f), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle run failed")
    return f


def run_window(f_window, nsteps, tau, force: Force, x0, y0, NX, NY):
    """nsteps steps of a window of a larger NX x NY periodic grid whose lower
    left cell is the global cell (x0, y0); only cells at least nsteps cells
    from the window's edges are valid afterwards (light cone)."""
    f = _f64(f_window).copy()
    _, wy, wx = f.shape
    rc = _load().orc_run_window(wx, wy, tau, force.ptr(), _p(f), int(nsteps), int(x0),
                                int(y0), int(NX), int(NY))
    if rc != 0:
        raise MemoryError("oracle window run failed")
    return f


def moments(f, force: Force = NO_FORCE):
    """Return dict rho, jx, jy, ux, uy (u = EDM velocity (j + F/2)/rho)."""
    f = _f64(f)
    _, ny, nx = f.shape
    out = {k: np.empty((ny, nx)) for k in ("rho", "jx", "jy", "ux", "uy")}
    _load().orc_moments(nx, ny, force.ptr(), _p(f), _p(out["rho"]), _p(out["jx"]),
                        _p(out["jy"]), _p(out["ux"]), _p(out["uy"]))
    return out


def ddx(A):
    A = _f64(A)
    ny, nx = A.shape
    out = np.empty_like(A)
    _load().orc_ddx(nx, ny, _p(A), _p(out))
    return out


def ddy(A):
    A = _f64(A)
    ny, nx = A.shape
    out = np.empty_like(A)
    _load().orc_ddy(nx, ny, _p(A), _p(out))
    return out


def bdf2(An, An1, An2):
    An, An1, An2 = _f64(An), _f64(An1), _f64(An2)
    out = np.empty_like(An)
    _load().orc_bdf2(An.size, _p(An), _p(An1), _p(An2), _p(out))
    return out


def terms(tau, rho3, ux3, uy3, Fx, Fy, nu=None):
    """13 term fields from (rho, u) at levels n, n-1, n-2 and F at n; the
    viscosity is (tau - 1/2)/3, or the per-cell field ``nu`` [ny, nx]."""
    rho3 = [_f64(a) for a in rho3]
    ux3 = [_f64(a) for a in ux3]
    uy3 = [_f64(a) for a in uy3]
    Fx, Fy = _f64(Fx), _f64(Fy)
    ny, nx = Fx.shape
    arr = (ctypes.c_void_p * 3)
    r = arr(*[a.ctypes.data for a in rho3])
    u = arr(*[a.ctypes.data for a in ux3])
    v = arr(*[a.ctypes.data for a in uy3])
    out = np.empty((NT, ny, nx))
    nu = None if nu is None else _f64(nu)
    rc = _load().orc_terms(nx, ny, tau, ctypes.cast(r, ctypes.c_void_p),
                           ctypes.cast(u, ctypes.c_void_p), ctypes.cast(v, ctypes.c_void_p),
                           _p(Fx), _p(Fy), None if nu is None else _p(nu), _p(out))
    if rc != 0:
        raise MemoryError("oracle terms failed")
    return out


def terms_from_populations(f_n, f_n1, f_n2, tau, force: Force = NO_FORCE):
    f_n, f_n1, f_n2 = _f64(f_n), _f64(f_n1), _f64(f_n2)
    _, ny, nx = f_n.shape
    out = np.empty((NT, ny, nx))
    rc = _load().orc_terms_from_populations(nx, ny, tau, force.ptr(), _p(f_n), _p(f_n1),
                                            _p(f_n2), _p(out))
    if rc != 0:
        raise MemoryError("oracle terms failed")
    return out


def box_mean(A, x0, y0, L):
    A = _f64(A)
    ny, nx = A.shape
    return _load().orc_box_mean(nx, ny, _p(A), int(x0), int(y0), int(L))


def box_values(terms13, x0, y0, L):
    terms13 = _f64(terms13)
    _, ny, nx = terms13.shape
    out = np.empty(NQ)
    _load().orc_box_values(nx, ny, _p(terms13), int(x0), int(y0), int(L), _p(out))
    return out


def balance_stats(terms13, Ls, origins=None, per_box=False):
    """Return stats[nL, 15, 2] (mean, population std) and optionally the
    per-box values [nL, n_boxes, 15]."""
    terms13 = _f64(terms13)
    _, ny, nx = terms13.shape
    Ls = np.ascontiguousarray(Ls, dtype=np.int32)
    nL = len(Ls)
    if origins is not None:
        origins = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1, 2)
        nb = origins.shape[0]
        op = _p(origins)
    else:
        nb = nx * ny
        op = None
    stats = np.empty((nL, NQ, 2))
    pb = np.empty((nL, nb, NQ)) if per_box else None
    rc = _load().orc_balance_stats(nx, ny, _p(terms13), _p(Ls), nL, op, nb, _p(stats),
                                   _p(pb) if per_box else None)
    if rc != 0:
        raise MemoryError("oracle stats failed")
    return (stats, pb) if per_box else stats


def box_mach(ux, uy, x0, y0, L):
    """Ma_V = sqrt(<|u|^2>_V) / c_s over the L x L box at (x0, y0), eq. (20)."""
    ux, uy = _f64(ux), _f64(uy)
    ny, nx = ux.shape
    return _load().orc_box_mach(nx, ny, _p(ux), _p(uy), int(x0), int(y0), int(L))


def hist_bin(v, edges):
    """Bin of v: the number of edges <= v (-1 for NaN)."""
    edges = _f64(edges)
    return _load().orc_bin(float(v), _p(edges), len(edges))


def distributions(terms13, ux, uy, Ls, delta_edges, mach_edges, origins=None):
    """Histograms over the boxes of each size of delta^E, delta^Omega
    ([nL, 2, len(delta_edges) + 1]) and of Ma_V ([nL, len(mach_edges) + 1]),
    and the mean and population std of Ma_V ([nL, 2])."""
    terms13, ux, uy = _f64(terms13), _f64(ux), _f64(uy)
    _, ny, nx = terms13.shape
    Ls = np.ascontiguousarray(Ls, dtype=np.int32)
    de, me = _f64(delta_edges), _f64(mach_edges)
    nL = len(Ls)
    if origins is not None:
        origins = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1, 2)
        nb, op = origins.shape[0], _p(origins)
    else:
        nb, op = nx * ny, None
    hd = np.zeros((nL, 2, len(de) + 1), dtype=np.int64)
    hm = np.zeros((nL, len(me) + 1), dtype=np.int64)
    ms = np.empty((nL, 2))
    rc = _load().orc_distributions(nx, ny, _p(terms13), _p(ux), _p(uy), _p(Ls), nL, op, nb,
                                   _p(de), len(de), _p(me), len(me), _p(hd), _p(hm), _p(ms))
    if rc != 0:
        raise MemoryError("oracle distributions failed")
    return hd, hm, ms


def global_quantities(f, tau, force: Force = NO_FORCE):
    """[sum rho, sum jx, sum jy, <E>, <Omega>, <u.F>, <eps>]."""
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.empty(7)
    rc = _load().orc_global(nx, ny, tau, force.ptr(), _p(f), _p(out))
    if rc != 0:
        raise MemoryError("oracle global failed")
    return out


def objective(f0, tau, force: Force, n0, n1, bx, by, L):
    """Mean over n in [n0, n1] of the L x L box average of RHS^{E,4}(n)."""
    f0 = _f64(f0)
    _, ny, nx = f0.shape
    J = ctypes.c_double()
    rc = _load().orc_objective(nx, ny, tau, force.ptr(), _p(f0), int(n0), int(n1),
                               int(bx), int(by), int(L), ctypes.byref(J))
    if rc != 0:
        raise MemoryError("oracle objective failed")
    return J.value


# --------------------------------------------------------------------------
# Three dimensions (D3Q19 and D3Q27; lbm_oracle3d.c).  Populations f[q, nz,
# ny, nx] (q = 19 or 27, read from the array's first axis), fields
# A[nz, ny, nx]; force = (kind, F0, kf, alpha) with kind 1 the cyclic
# Kolmogorov force F0 (sin(2 pi kf y/ny), sin(2 pi kf z/nz), sin(2 pi kf x/nx)).
# --------------------------------------------------------------------------

def _q3(q):
    if q not in (19, 27):
        raise ValueError("3D lattice must be D3Q19 or D3Q27")
    return q


def lattice3(q=19):
    q = _q3(q)
    cx, cy, cz = (np.zeros(q, np.int32) for _ in range(3))
    t = np.zeros(q)
    _load().orc3_lattice(q, _p(cx), _p(cy), _p(cz), _p(t))
    return cx, cy, cz, t


def feq3(rho, ux, uy, uz, q=19):
    q = _q3(q)
    out = np.zeros(q)
    _load().orc3_feq(q, float(rho), float(ux), float(uy), float(uz), _p(out))
    return out


def init3(rho, ux, uy, uz, q=19):
    q = _q3(q)
    rho, ux, uy, uz = (_f64(a) for a in (rho, ux, uy, uz))
    nz, ny, nx = rho.shape
    f = np.empty((q, nz, ny, nx))
    _load().orc3_init(q, nx, ny, nz, _p(rho), _p(ux), _p(uy), _p(uz), _p(f))
    return f


def run3(f, nsteps, tau, kind=0, F0=0.0, kf=0, alpha=0.0):
    f = _f64(f).copy()
    q, nz, ny, nx = f.shape
    if _load().orc3_run(_q3(q), nx, ny, nz, float(tau), int(kind), float(F0), int(kf),
                        float(alpha), _p(f), int(nsteps)) != 0:
        raise MemoryError("oracle 3D run failed")
    return f


def moments3(f, kind=0, F0=0.0, kf=0, alpha=0.0):
    """dict rho, ux, uy, uz (u = (j + F/2)/rho), Fx, Fy, Fz (F = F_ext - alpha j)."""
    f = _f64(f)
    q, nz, ny, nx = f.shape
    out = {k: np.empty((nz, ny, nx)) for k in ("rho", "ux", "uy", "uz", "Fx", "Fy", "Fz")}
    _load().orc3_moments(_q3(q), nx, ny, nz, int(kind), float(F0), int(kf), float(alpha), _p(f),
                         *(_p(out[k]) for k in ("rho", "ux", "uy", "uz", "Fx", "Fy", "Fz")))
    return out


def d3(A, axis):
    """Eq. (18) along axis 0 = x, 1 = y, 2 = z of A[nz, ny, nx]."""
    A = _f64(A)
    nz, ny, nx = A.shape
    out = np.empty_like(A)
    _load().orc3_d(nx, ny, nz, int(axis), _p(A), _p(out))
    return out


def terms3(tau, rho3, ux3, uy3, uz3, Fx, Fy, Fz):
    """13 term fields [13, nz, ny, nx] from (rho, u) at n, n-1, n-2 and F at n."""
    levels = [[_f64(a) for a in L] for L in (rho3, ux3, uy3, uz3)]
    Fx, Fy, Fz = _f64(Fx), _f64(Fy), _f64(Fz)
    nz, ny, nx = Fx.shape
    arr = ctypes.c_void_p * 3
    ptrs = [arr(*[a.ctypes.data for a in L]) for L in levels]
    out = np.empty((NT, nz, ny, nx))
    rc = _load().orc3_terms(nx, ny, nz, float(tau), *(ctypes.cast(p, ctypes.c_void_p) for p in ptrs),
                            _p(Fx), _p(Fy), _p(Fz), _p(out))
    if rc != 0:
        raise MemoryError("oracle 3D terms failed")
    return out


def terms3_from_populations(f_n, f_n1, f_n2, tau, kind=0, F0=0.0, kf=0, alpha=0.0):
    f_n, f_n1, f_n2 = _f64(f_n), _f64(f_n1), _f64(f_n2)
    q, nz, ny, nx = f_n.shape
    assert f_n1.shape == f_n.shape and f_n2.shape == f_n.shape
    out = np.empty((NT, nz, ny, nx))
    rc = _load().orc3_terms_from_populations(_q3(q), nx, ny, nz, float(tau), int(kind), float(F0),
                                             int(kf), float(alpha), _p(f_n), _p(f_n1), _p(f_n2),
                                             _p(out))
    if rc != 0:
        raise MemoryError("oracle 3D terms failed")
    return out


def box_mean3(A, x0, y0, z0, L):
    A = _f64(A)
    nz, ny, nx = A.shape
    return _load().orc3_box_mean(nx, ny, nz, _p(A), int(x0), int(y0), int(z0), int(L))


def balance_stats3(T, Ls, origins=None, per_box=False):
    """stats [nL, 15, 2] (and per-box [nL, boxes, 15]) of L^3 boxes; origins
    None (every periodic origin) or [n, 3] (x0, y0, z0) triples."""
    T = _f64(T)
    _, nz, ny, nx = T.shape
    Ls = np.ascontiguousarray(Ls, dtype=np.int32)
    if origins is not None:
        origins = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1, 3)
        nb, op = origins.shape[0], _p(origins)
    else:
        nb, op = nx * ny * nz, None
    stats = np.empty((len(Ls), NQ, 2))
    pb = np.empty((len(Ls), nb, NQ)) if per_box else None
    rc = _load().orc3_balance_stats(nx, ny, nz, _p(T), _p(Ls), len(Ls), op, nb, _p(stats),
                                    _p(pb) if per_box else None)
    if rc != 0:
        raise MemoryError("oracle 3D stats failed")
    return (stats, pb) if per_box else stats
