"""GB300 (sm_103a) D2Q9 lattice Boltzmann library with the sub-volume
energy/enstrophy balance diagnostic of Tauzin et al. (2018).

This module is a thin binding of the C ABI in ``include/lbm.h``: it marshals
arguments and lets PyTorch provide device memory (the workspace) and the CUDA
stream.  Every step of the method runs in the CUDA kernels of ``liblbm.so``;
there is no Python or CPU fallback, and the import fails loudly when the
library has not been built (``python -m paper_1809_06735_gb300.build`` or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

LBM_OK = 0
ERRORS = {-1: "invalid argument", -2: "workspace", -3: "CUDA error", -4: "history missing",
          -5: "member diverged", -6: "timeout"}
NTERMS = 13
NQUANT = 15
NGLOBAL = 7
TERM_NAMES = ["LHS_E", "RHS_E1", "RHS_E2", "RHS_E3", "RHS_E4", "RHS_E5",
              "LHS_Z", "RHS_Z1", "RHS_Z2", "RHS_Z3", "RHS_Z4", "RHS_Z5", "RHS_Z6"]
QUANTITY_NAMES = ["delta_E", "delta_Z"] + TERM_NAMES
GLOBAL_NAMES = ["mass", "jx", "jy", "E", "Omega", "uF", "eps"]


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lbm error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _MemberCfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("tau", ctypes.c_double),
                ("rho0", ctypes.c_double), ("force_kind", ctypes.c_int), ("kf", ctypes.c_int),
                ("F0", ctypes.c_double), ("alpha", ctypes.c_double),
                ("phase", ctypes.c_double), ("FR0", ctypes.c_double),
                ("collision", ctypes.c_int), ("Cs", ctypes.c_double)]


class _MemberCfg3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("force_kind", ctypes.c_int), ("kf", ctypes.c_int), ("F0", ctypes.c_double),
                ("alpha", ctypes.c_double)]


class _Config3(ctypes.Structure):
    _fields_ = [("n_members", ctypes.c_int), ("members", ctypes.POINTER(_MemberCfg3)),
                ("precision", ctypes.c_int), ("diag_every", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p), ("lattice", ctypes.c_int),
                ("diag_precision", ctypes.c_int)]


class _Config(ctypes.Structure):
    _fields_ = [("n_members", ctypes.c_int), ("members", ctypes.POINTER(_MemberCfg)),
                ("precision", ctypes.c_int), ("storage", ctypes.c_int),
                ("diag_every", ctypes.c_int), ("graph_steps", ctypes.c_int),
                ("diag_precision", ctypes.c_int), ("diag_batch", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load ``liblbm.so`` and declare the C signatures.  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblbm.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    I, P, D, S = ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_size_t
    sig = {
        "lbm_workspace_size": ([ctypes.POINTER(_Config), ctypes.POINTER(S)], I),
        "lbm_create": ([ctypes.POINTER(_Config), P, S, ctypes.POINTER(P)], I),
        "lbm_destroy": ([P], I),
        "lbm_init_fields": ([P, I, P, P, P, I], I),
        "lbm_init_fields_batch": ([P, P, I, P, P, P, I], I),
        "lbm_step": ([P, I], I),
        "lbm_time": ([P], ctypes.c_longlong),
        "lbm_launch_count": ([P], ctypes.c_longlong),
        "lbm_kernels_per_step": ([P], ctypes.c_longlong),
        "lbm_set_launch": ([P, I, I, I, I], I),
        "lbm_tuning": ([P, P, P, P, P, P, P], I),
        "lbm_record_snapshot": ([P], I),
        "lbm_moments": ([P, I, P, P, P, P], I),
        "lbm_global_balance": ([P, I, P], I),
        "lbm_subvolume_balance": ([P, I, P, I, P, P, P, P], I),
        "lbm_subvolume_balance_batch": ([P, P, I, P, I, P, P, P], I),
        "lbm_subvolume_balance_async": ([P, P, I, P, I, P, P, P], I),
        "lbm_subvolume_distributions": ([P, P, I, P, I, P, P, P, I, P, I, P, P, P, P], I),
        "lbm_diag_synchronize": ([P], I),
        "lbm_get_populations": ([P, I, P, I], I),
        "lbm_set_populations": ([P, I, P, I], I),
        "lbm_member_status": ([P, I, P], I),
        "lbm_adjoint_step": ([P, I, P, P, P, D, I, I, I, P, P], I),
        "lbm_objective_accumulate": ([P, I, D, I, I, I, P], I),
        "lbm_objective_steps": ([P, I, I, D, I, I, I, P], I),
        "lbm_record_trajectory": ([P, I, I, P], I),
        "lbm_adjoint_sweep": ([P, I, P, I, P, P, P, P, I, I, I, P, P], I),
        "lbm_last_error": ([P], ctypes.c_char_p),
        "lbm_probe_fma_rate": ([I, P, P], I),
        "lbm_probe_grid_barrier": ([I, I, I, P, P], I),
        "lbm3d_workspace_size": ([ctypes.POINTER(_Config3), ctypes.POINTER(S)], I),
        "lbm3d_create": ([ctypes.POINTER(_Config3), P, S, ctypes.POINTER(P)], I),
        "lbm3d_destroy": ([P], I),
        "lbm3d_init_fields": ([P, I, P, P, P, P, I], I),
        "lbm3d_step": ([P, I], I),
        "lbm3d_time": ([P], ctypes.c_longlong),
        "lbm3d_cells_per_lane": ([P], I),
        "lbm3d_set_cells_per_lane": ([P, I], I),
        "lbm3d_get_populations": ([P, I, P, I], I),
        "lbm3d_set_populations": ([P, I, P, I], I),
        "lbm3d_record_snapshot": ([P], I),
        "lbm3d_subvolume_balance": ([P, I, P, I, P, P, P, P], I),
        "lbm3d_last_error": ([P], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


@dataclass
class Member:
    """One ensemble member: an nx x ny doubly periodic grid with relaxation
    time tau (eq. (1), nu = (tau - 1/2)/3 by eq. (5)), reference density rho0,
    an optional force -- kind 1: Kolmogorov F0 (sin(2 pi kf y/ny),
    sin(2 pi kf x/nx)); kind 2: the paper's shell force of eqs. (14), (15)
    (amplitude F0, phase) with the large-scale damping of eq. (16) (FR0) --
    linear drag alpha on the bare momentum, and the collision: 0 BGK, 1
    Smagorinsky (constant Cs), 2 the turbulent viscosity of eq. (7), 3 the
    entropic LBM."""
    nx: int
    ny: int
    tau: float
    rho0: float = 1.0
    force_kind: int = 0
    kf: int = 0
    F0: float = 0.0
    alpha: float = 0.0
    phase: float = 0.0
    FR0: float = 0.0
    collision: int = 0
    Cs: float = 0.0

    def c(self) -> _MemberCfg:
        return _MemberCfg(self.nx, self.ny, self.tau, self.rho0, self.force_kind, self.kf,
                          self.F0, self.alpha, self.phase, self.FR0, self.collision, self.Cs)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous(), "tensors passed to the library must be contiguous"
    return t.data_ptr()


class Lattice:
    """A handle over a batch of members sharing precision and stream.

    ``precision`` 32 stores FP32 deviations f - t rho0 (batched vector kernel),
    64 stores plain FP64 populations.  The workspace is one torch uint8 CUDA
    tensor sized by ``lbm_workspace_size``; all work goes to ``stream``
    (default: the current torch stream at construction)."""

    def __init__(self, members: Sequence[Member], precision: int = 32, diag_every: int = 0,
                 graph_steps: int = 0, stream=None, device=None, diag_precision: int = 0,
                 storage: int = 0, diag_batch: int = 0):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.members = list(members)
        self.precision = precision
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        arr = (_MemberCfg * len(self.members))(*[m.c() for m in self.members])
        self._arr = arr
        self._cfg = _Config(len(self.members), arr, precision, storage, diag_every, graph_steps,
                            diag_precision, diag_batch, ctypes.c_void_p(self.stream.cuda_stream))
        nbytes = ctypes.c_size_t()
        self._check(self.lib.lbm_workspace_size(ctypes.byref(self._cfg), ctypes.byref(nbytes)))
        self.workspace_bytes = nbytes.value
        self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8,
                                     device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._check(self.lib.lbm_create(ctypes.byref(self._cfg), ctypes.c_void_p(aligned),
                                            self.workspace_bytes, ctypes.byref(h)))
        self.h = h

    # -- plumbing -------------------------------------------------------
    def _check(self, rc: int):
        if rc != LBM_OK:
            h = getattr(self, "h", None)
            msg = self.lib.lbm_last_error(h).decode()
            raise LBMError(rc, msg)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.lbm_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, dtype=None):
        torch = self._torch
        dtype = dtype or torch.float64
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a))
        return a.to(device=self.device, dtype=dtype).contiguous()

    def _shape(self, m):
        return self.members[m].ny, self.members[m].nx

    # -- state ------------------------------------------------------------
    def init_fields(self, member: int, rho, ux, uy):
        """f(x, 0) = f_eq(rho(x), u(x)).  numpy arrays are passed as host
        pointers (the library copies them), tensors as device pointers."""
        if isinstance(rho, np.ndarray):
            r, u, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
            self._check(self.lib.lbm_init_fields(self.h, member, _ptr(r), _ptr(u), _ptr(v), 0))
        else:
            r, u, v = (self._dev(a) for a in (rho, ux, uy))
            self._check(self.lib.lbm_init_fields(self.h, member, _ptr(r), _ptr(u), _ptr(v), 1))
            self._keep = (r, u, v)

    def init_fields_batch(self, members, rho, ux, uy):
        """init_fields for several members (equal grids) from stacked fields
        [n, ny, nx]: numpy arrays go through one host copy per field and a
        single synchronisation; CPU tensors are passed as host pointers
        (pinned ones are read in place by the kernel, asynchronously: keep
        them unchanged until the stream has passed the call); CUDA tensors
        are read on the device."""
        mem = np.ascontiguousarray(members, dtype=np.int32)
        if isinstance(rho, np.ndarray):
            r, u, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
            on_dev = 0
        elif not rho.is_cuda:
            r, u, v = rho, ux, uy
            for a in (r, u, v):
                assert a.dtype == self._torch.float64 and a.is_contiguous()
            on_dev = 0
            self._keep = (r, u, v)
        else:
            r, u, v = (self._dev(a) for a in (rho, ux, uy))
            on_dev = 1
            self._keep = (r, u, v)
        for a in (r, u, v):
            assert a.shape[0] == len(mem), "one field block per listed member"
        self._check(self.lib.lbm_init_fields_batch(self.h, _ptr(mem), len(mem), _ptr(r), _ptr(u),
                                                   _ptr(v), on_dev))

    def step(self, nsteps: int = 1):
        self._check(self.lib.lbm_step(self.h, int(nsteps)))

    @property
    def time(self) -> int:
        return int(self.lib.lbm_time(self.h))

    @property
    def launch_count(self) -> int:
        """Kernels issued by this handle so far (graph nodes counted)."""
        return int(self.lib.lbm_launch_count(self.h))

    def tuning(self) -> dict:
        """Launch configuration in use (storage 'aa' or 'double_buffer', CTA
        shape, grid, autotuned ms per step, kernels per time step)."""
        st, w, r, g, pr = (ctypes.c_int() for _ in range(5))
        ms = ctypes.c_float()
        self._check(self.lib.lbm_tuning(self.h, ctypes.byref(st), ctypes.byref(w), ctypes.byref(r),
                                        ctypes.byref(g), ctypes.byref(ms), ctypes.byref(pr)))
        return {"storage": "aa" if st.value == 1 else "double_buffer", "warps_per_cta": w.value,
                "rows_per_warp": r.value, "grid_ctas": g.value, "tuned_step_ms": ms.value,
                "projection_rows": pr.value,
                "kernels_per_step": int(self.lib.lbm_kernels_per_step(self.h))}

    def set_launch(self, warps: int, rows: int, grid: int = 0, proj_rows: int = 0):
        """Replace the autotuned launch configuration (see lbm_set_launch);
        proj_rows 0 keeps the projection's rows per thread."""
        self._check(self.lib.lbm_set_launch(self.h, warps, rows, grid, proj_rows))

    def record_snapshot(self):
        self._check(self.lib.lbm_record_snapshot(self.h))

    def get_populations(self, member: int, out=None):
        """Public pre-collision populations f[9, ny, nx] (float64, device)."""
        ny, nx = self._shape(member)
        if out is None:
            out = self._torch.empty((9, ny, nx), dtype=self._torch.float64, device=self.device)
        self._check(self.lib.lbm_get_populations(self.h, member, _ptr(out), 1))
        return out

    def get_populations_host(self, member: int) -> np.ndarray:
        ny, nx = self._shape(member)
        out = np.empty((9, ny, nx))
        self._check(self.lib.lbm_get_populations(self.h, member, _ptr(out), 0))
        return out

    def set_populations(self, member: int, f):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
            self._check(self.lib.lbm_set_populations(self.h, member, _ptr(f), 0))
        else:
            f = self._dev(f)
            self._check(self.lib.lbm_set_populations(self.h, member, _ptr(f), 1))
            self._keep_f = f

    def member_status(self, member: int) -> int:
        s = ctypes.c_int()
        self._check(self.lib.lbm_member_status(self.h, member, ctypes.byref(s)))
        return s.value

    # -- diagnostics ------------------------------------------------------
    def moments(self, member: int):
        """rho, u = (j + F/2)/rho and omega (eq. (18)) as float64 device tensors."""
        torch = self._torch
        ny, nx = self._shape(member)
        out = {k: torch.empty((ny, nx), dtype=torch.float64, device=self.device)
               for k in ("rho", "ux", "uy", "omega")}
        self._check(self.lib.lbm_moments(self.h, member, _ptr(out["rho"]), _ptr(out["ux"]),
                                         _ptr(out["uy"]), _ptr(out["omega"])))
        return out

    def global_balance(self, member: int) -> np.ndarray:
        out = np.empty(NGLOBAL)
        self._check(self.lib.lbm_global_balance(self.h, member, _ptr(out)))
        return out

    @staticmethod
    def _origin_lists(Ls, origins):
        """(concatenated origins [n, 2] int32, counts [nL] int32) or (None, None).
        ``origins``: None (all periodic origins), one [n, 2] array used for
        every size, or a sequence of nL arrays (one per size)."""
        if origins is None:
            return None, None
        if isinstance(origins, np.ndarray) or (len(origins) and np.isscalar(origins[0][0])):
            o = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1, 2)
            per = [o] * len(Ls)
        else:
            per = [np.ascontiguousarray(o, dtype=np.int32).reshape(-1, 2) for o in origins]
            if len(per) != len(Ls):
                raise ValueError("one origin array per box size is required")
        counts = np.array([p.shape[0] for p in per], dtype=np.int32)
        return np.ascontiguousarray(np.concatenate(per, axis=0)), counts

    def subvolume_balance(self, member: int, Ls, origins=None, per_box: bool = False):
        """Statistics [nL, 15, 2] (mean, population std) of the box quantities
        [delta^E, delta^Omega, 13 terms]; with ``per_box`` also the device
        tensor of every box, [rows, 15] in the order of Ls (rows = nL * nx * ny
        for all origins).  ``origins``: see ``_origin_lists``."""
        Ls = np.ascontiguousarray(Ls, dtype=np.int32)
        nL = len(Ls)
        ny, nx = self._shape(member)
        o, counts = self._origin_lists(Ls, origins)
        rows = nL * nx * ny if o is None else int(counts.sum())
        stats = np.empty((nL, NQUANT, 2))
        pb = None
        if per_box:
            pb = self._torch.empty((rows, NQUANT), dtype=self._torch.float64,
                                   device=self.device)
        self._check(self.lib.lbm_subvolume_balance(
            self.h, member, _ptr(Ls), nL, _ptr(o), _ptr(counts), _ptr(stats), _ptr(pb)))
        return (stats, pb) if per_box else stats

    def subvolume_balance_batch(self, members, Ls, origins=None):
        """Statistics [n_members, nL, 15, 2] for several members, one sync."""
        mem = np.ascontiguousarray(members, dtype=np.int32)
        Ls = np.ascontiguousarray(Ls, dtype=np.int32)
        stats = np.empty((len(mem), len(Ls), NQUANT, 2))
        o, counts = self._origin_lists(Ls, origins)
        self._check(self.lib.lbm_subvolume_balance_batch(
            self.h, _ptr(mem), len(mem), _ptr(Ls), len(Ls), _ptr(o), _ptr(counts), _ptr(stats)))
        return stats

    def subvolume_distributions(self, members, Ls, delta_edges, mach_edges, origins=None):
        """Distributions over the boxes of each size (one sync): a dict with
        ``stats`` [n, nL, 15, 2] (as ``subvolume_balance_batch``),
        ``delta_hist`` [n, nL, 2, len(delta_edges) + 1] box counts of
        delta^E, delta^Omega per bin, ``mach_hist`` [n, nL, len(mach_edges) + 1]
        and ``mach`` [n, nL, 2] (mean, std) of the sub-volume Mach number
        Ma_V = sqrt(<|u|^2>_V) / c_s.  Bin b holds edges[b-1] <= v < edges[b]."""
        mem = np.ascontiguousarray(members, dtype=np.int32)
        Ls = np.ascontiguousarray(Ls, dtype=np.int32)
        de = np.ascontiguousarray(delta_edges, dtype=np.float64)
        me = np.ascontiguousarray(mach_edges, dtype=np.float64)
        n, nL = len(mem), len(Ls)
        stats = np.empty((n, nL, NQUANT, 2))
        dh = np.empty((n, nL, 2, len(de) + 1), dtype=np.int64)
        mh = np.empty((n, nL, len(me) + 1), dtype=np.int64)
        ma = np.empty((n, nL, 2))
        o, counts = self._origin_lists(Ls, origins)
        self._check(self.lib.lbm_subvolume_distributions(
            self.h, _ptr(mem), n, _ptr(Ls), nL, _ptr(o), _ptr(counts), _ptr(de), len(de),
            _ptr(me), len(me), _ptr(stats), _ptr(dh), _ptr(mh), _ptr(ma)))
        return {"stats": stats, "delta_hist": dh, "mach_hist": mh, "mach": ma}

    def subvolume_balance_async(self, members, Ls, origins=None, out=None):
        """Queue the diagnostic of the current time on the handle's diagnostic
        stream and return at once; statistics land in the device tensor
        ``out`` [n_members, nL, 15, 2] (allocated when None) once the work is
        done (``diag_synchronize`` or any later ordered call)."""
        mem = np.ascontiguousarray(members, dtype=np.int32)
        Ls = np.ascontiguousarray(Ls, dtype=np.int32)
        if out is None:
            out = self._torch.empty((len(mem), len(Ls), NQUANT, 2), dtype=self._torch.float64,
                                    device=self.device)
        o, counts = self._origin_lists(Ls, origins)
        self._check(self.lib.lbm_subvolume_balance_async(
            self.h, _ptr(mem), len(mem), _ptr(Ls), len(Ls), _ptr(o), _ptr(counts), _ptr(out)))
        return out

    def diag_synchronize(self):
        self._check(self.lib.lbm_diag_synchronize(self.h))

    # -- adjoint ------------------------------------------------------------
    def adjoint_step(self, member: int, f_n, lam_in, lam_out, weight: float, box, L: int,
                     dJ_dtau, dJ_dF0):
        """lam_out = (dS/df)^T lam_in + weight * dJ_n/df at the state f_n; adds
        the parameter gradients of this step into dJ_dtau, dJ_dF0 (device
        float64 scalars)."""
        self._check(self.lib.lbm_adjoint_step(self.h, member, _ptr(f_n), _ptr(lam_in),
                                              _ptr(lam_out), float(weight), int(box[0]),
                                              int(box[1]), int(L), _ptr(dJ_dtau),
                                              _ptr(dJ_dF0)))

    def objective_accumulate(self, member: int, weight: float, box, L: int, acc):
        """acc += weight * (L x L box average of RHS^{E,4} at the current time)."""
        self._check(self.lib.lbm_objective_accumulate(self.h, member, float(weight),
                                                      int(box[0]), int(box[1]), int(L),
                                                      _ptr(acc)))

    def objective_steps(self, member: int, nsteps: int, weight: float, box, L: int, acc):
        """nsteps times: acc += weight * (box average at the current time), then
        one step of every member."""
        self._check(self.lib.lbm_objective_steps(self.h, member, int(nsteps), float(weight),
                                                 int(box[0]), int(box[1]), int(L), _ptr(acc)))

    def record_trajectory(self, member: int, states):
        """states[k] = public state at the current time + k (device tensor
        [nstates, 9, ny, nx] float64), stepping nstates - 1 times."""
        assert states.dtype == self._torch.float64 and states.is_cuda
        self._check(self.lib.lbm_record_trajectory(self.h, member, int(states.shape[0]),
                                                   _ptr(states)))

    def adjoint_sweep(self, member: int, states, lam_in, lam_out, lam_tmp, weights, box,
                      L: int, dJ_dtau, dJ_dF0):
        """Adjoint steps over the levels of ``states`` (last to first), from
        lam_in = dJ/df(after the last level; None for zero) to lam_out =
        dJ/df(first level); ``weights`` holds the objective weight of each
        level; parameter gradients added into dJ_dtau, dJ_dF0."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        assert w.shape == (states.shape[0],)
        self._check(self.lib.lbm_adjoint_sweep(self.h, member, _ptr(states), int(states.shape[0]),
                                               _ptr(lam_in), _ptr(lam_out), _ptr(lam_tmp),
                                               _ptr(w), int(box[0]), int(box[1]), int(L),
                                               _ptr(dJ_dtau), _ptr(dJ_dF0)))


def probe_fma_rate(bits: int, stream=None) -> float:
    """Measured FMA throughput of the device in flop/s (bits 64 or 32)."""
    lib = load_library()
    out = ctypes.c_double()
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = lib.lbm_probe_fma_rate(int(bits), s, ctypes.byref(out))
    if rc != LBM_OK:
        raise LBMError(rc, lib.lbm_last_error(None).decode())
    return out.value


def probe_grid_barrier(ctas: int, rounds: int, withhold: int = -1, stream=None) -> int:
    """Runs the persistent step's grid barrier alone; returns 1 if the CTAs
    gave up waiting (CTA ``withhold`` never arriving), else 0."""
    lib = load_library()
    out = ctypes.c_int(-1)
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = lib.lbm_probe_grid_barrier(int(ctas), int(rounds), int(withhold), s, ctypes.byref(out))
    if rc != LBM_OK:
        raise LBMError(rc, lib.lbm_last_error(None).decode())
    return out.value


def workspace_size(members: Sequence[Member], precision: int = 32, diag_every: int = 0,
                   graph_steps: int = 0, diag_batch: int = 0) -> int:
    """Host-only query of the device workspace bytes for a configuration."""
    lib = load_library()
    arr = (_MemberCfg * len(members))(*[m.c() for m in members])
    cfg = _Config(len(members), arr, precision, 0, diag_every, graph_steps, 0, diag_batch, None)
    n = ctypes.c_size_t()
    rc = lib.lbm_workspace_size(ctypes.byref(cfg), ctypes.byref(n))
    if rc != LBM_OK:
        raise LBMError(rc, lib.lbm_last_error(None).decode())
    return n.value


@dataclass
class Member3:
    """One member of the three-dimensional extension: an nx x ny x nz doubly
    periodic D3Q19 grid, relaxation time tau, reference density rho0, the
    cyclic Kolmogorov force F0 (sin(2 pi kf y/ny), sin(2 pi kf z/nz),
    sin(2 pi kf x/nx)) when force_kind == 1, drag alpha."""
    nx: int
    ny: int
    nz: int
    tau: float
    rho0: float = 1.0
    force_kind: int = 0
    kf: int = 0
    F0: float = 0.0
    alpha: float = 0.0

    def c(self) -> _MemberCfg3:
        return _MemberCfg3(self.nx, self.ny, self.nz, self.tau, self.rho0, self.force_kind,
                           self.kf, self.F0, self.alpha)


class Lattice3D:
    """Handle over D3Q19 or D3Q27 members (``lattice`` 19 or 27;
    include/lbm3d.h): FP32 deviation or FP64 storage, balance terms in FP64
    (``diag_precision`` 0 or 64) or FP32 (32), workspace in one torch uint8
    CUDA tensor, work on ``stream``."""

    def __init__(self, members: Sequence[Member3], precision: int = 32, diag_every: int = 0,
                 stream=None, device=None, lattice: int = 19, diag_precision: int = 0):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.members = list(members)
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._arr = (_MemberCfg3 * len(self.members))(*[m.c() for m in self.members])
        self.q = 27 if lattice == 27 else 19
        self._cfg = _Config3(len(self.members), self._arr, precision, diag_every,
                             ctypes.c_void_p(self.stream.cuda_stream), int(lattice),
                             int(diag_precision))
        n = ctypes.c_size_t()
        self._check(self.lib.lbm3d_workspace_size(ctypes.byref(self._cfg), ctypes.byref(n)))
        self.workspace = torch.empty(n.value + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._check(self.lib.lbm3d_create(ctypes.byref(self._cfg), ctypes.c_void_p(aligned),
                                              n.value, ctypes.byref(h)))
        self.h = h

    def _check(self, rc: int):
        if rc != LBM_OK:
            msg = self.lib.lbm3d_last_error(getattr(self, "h", None)).decode()
            raise LBMError(rc, msg)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.lbm3d_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self, m):
        M = self.members[m]
        return M.nz, M.ny, M.nx

    def init_fields(self, member: int, rho, ux, uy, uz):
        """f(x, 0) = f_eq(rho, u) from host arrays [nz, ny, nx]."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy, uz)]
        self._check(self.lib.lbm3d_init_fields(self.h, member, *[_ptr(a) for a in arrs], 0))

    def step(self, nsteps: int = 1):
        self._check(self.lib.lbm3d_step(self.h, int(nsteps)))

    @property
    def time(self) -> int:
        return int(self.lib.lbm3d_time(self.h))

    def tuning(self) -> dict:
        """Cells per lane of the vectorised FP32 kernel (4 or 2, timed at
        create; 0 when no member takes it)."""
        return {"cells_per_lane": int(self.lib.lbm3d_cells_per_lane(self.h))}

    def set_cells_per_lane(self, cpl: int):
        """4 or 2 cells per lane in the vectorised FP32 kernel."""
        self._check(self.lib.lbm3d_set_cells_per_lane(self.h, int(cpl)))

    def record_snapshot(self):
        self._check(self.lib.lbm3d_record_snapshot(self.h))

    def get_populations_host(self, member: int) -> np.ndarray:
        out = np.empty((self.q,) + self._shape(member))
        self._check(self.lib.lbm3d_get_populations(self.h, member, _ptr(out), 0))
        return out

    def set_populations(self, member: int, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        self._check(self.lib.lbm3d_set_populations(self.h, member, _ptr(f), 0))

    def subvolume_balance(self, member: int, Ls, origins=None, per_box: bool = False):
        """Statistics [nL, 15, 2] over L^3 boxes (every periodic origin, or one
        [n, 3] array of (x0, y0, z0) per size); with ``per_box`` also the
        device tensor [rows, 15]."""
        Ls = np.ascontiguousarray(Ls, dtype=np.int32)
        nz, ny, nx = self._shape(member)
        o = counts = None
        if origins is not None:
            per = [np.ascontiguousarray(a, dtype=np.int32).reshape(-1, 3) for a in origins]
            counts = np.array([p.shape[0] for p in per], dtype=np.int32)
            o = np.ascontiguousarray(np.concatenate(per, 0))
        rows = len(Ls) * nx * ny * nz if o is None else int(counts.sum())
        stats = np.empty((len(Ls), NQUANT, 2))
        pb = None
        if per_box:
            pb = self._torch.empty((rows, NQUANT), dtype=self._torch.float64, device=self.device)
        self._check(self.lib.lbm3d_subvolume_balance(self.h, member, _ptr(Ls), len(Ls), _ptr(o),
                                                     _ptr(counts), _ptr(stats), _ptr(pb)))
        return (stats, pb) if per_box else stats
