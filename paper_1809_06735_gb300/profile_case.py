"""Small, self-contained runs of each kernel family for Nsight Compute.

    python -m paper_1809_06735_gb300.profile_case step     # batched FP32 stream-collide
    python -m paper_1809_06735_gb300.profile_case step_full  # the same, 64 x 512^2
    python -m paper_1809_06735_gb300.profile_case diag     # one diagnostic event, 512^2
    python -m paper_1809_06735_gb300.profile_case diag_batch  # batched event, 16 x 512^2
    python -m paper_1809_06735_gb300.profile_case paper_forcing  # force kind 2, 64 x 256^2
    python -m paper_1809_06735_gb300.profile_case collisions  # Smagorinsky, eq. (7), ELBM
    python -m paper_1809_06735_gb300.profile_case 3d       # D3Q19, 2 x 128^3; 3D balance
    python -m paper_1809_06735_gb300.profile_case fp64     # plain FP64 step, 512^2
    python -m paper_1809_06735_gb300.profile_case adjoint  # FP64 adjoint steps, 256^2

Sizes keep the working set above the L2 (so DRAM counters mean something)
and below a few GB.  The step case creates its handle with the launch-shape
autotuner on: 2 storages x 18 shapes x 8 launches = 288 launches of k_step_f32_vec come
before the first step of the run.
"""
from __future__ import annotations

import sys

import numpy as np
import torch

import lbm_inputs as li

from . import Lattice, Member

AUTOTUNE_LAUNCHES = 288


def case_step(members=16, n=512, steps=25):
    lat = Lattice([Member(n, n, 0.52)] * members, precision=32, graph_steps=0)
    for m in range(members):
        lat.init_fields(m, *li.random_phase(n, seed=1000 + m, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("step case done:", lat.launch_count, "launches")


def case_step_full(members=64, n=512, steps=200):
    """The ensemble benchmark's stream-collide workload (64 x 512^2, FP32,
    autotuned storage and shape) for single-pass DRAM counters; the
    autotuner's 288 launches and the 64 initialisations come first."""
    lat = Lattice([Member(n, n, 0.52)] * members, precision=32, graph_steps=0, diag_batch=1)
    for m in range(members):
        lat.init_fields(m, *li.random_phase(n, seed=1000 + m, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("step_full case done:", lat.launch_count, "launches", lat.tuning())


def case_paper_forcing(members=64, n=256, steps=30):
    """The paper's forcing (force kind 2) on 64 FP32 members of 256^2: the
    damping projection and the stream-collide with the shell-force table."""
    lat = Lattice([Member(n, n, 0.52, 1.0, 2, 0, 8e-4, 0.0, 0.0, 1e-5)] * members,
                  precision=32, graph_steps=0)
    for m in range(members):
        lat.init_fields(m, *li.random_phase(n, seed=3000 + m, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("paper forcing case done:", lat.launch_count, "launches", lat.tuning())


def case_collisions(members=16, n=512, steps=12):
    """The variable-viscosity collisions on 16 FP32 members of 512^2: one
    handle each for Smagorinsky, eq. (7) and the entropic LBM."""
    fields = li.random_phase(n, seed=4000, u_rms=0.02)
    for coll, cs in ((1, 0.1), (2, 0.0), (3, 0.0)):
        lat = Lattice([Member(n, n, 0.51, collision=coll, Cs=cs)] * members, precision=32,
                      graph_steps=0)
        for m in range(members):
            lat.init_fields(m, *fields)
        lat.step(steps)
        torch.cuda.synchronize()
        print("collision", coll, "done:", lat.launch_count, "launches", lat.tuning())
        del lat


def case_3d(members=2, n=128, steps=12):
    """The D3Q19 and D3Q27 stream-collide on 2 FP32 members of 128^3 each,
    then one FP64 balance event on a 48^3 member."""
    from . import Lattice3D, Member3
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ux, uy = 0.02 * np.sin(X) * np.cos(Y) * np.cos(Z), -0.02 * np.cos(X) * np.sin(Y) * np.cos(Z)
    uz, rho = 0.005 * np.sin(X - Y), np.ones((n, n, n))
    for q in (19, 27):
        lat = Lattice3D([Member3(n, n, n, 0.52)] * members, precision=32, lattice=q)
        for m in range(members):
            lat.init_fields(m, rho, ux, uy, uz)
        lat.step(steps)
        torch.cuda.synchronize()
        del lat
    nd = 48
    dl = Lattice3D([Member3(nd, nd, nd, 0.52)], precision=64, diag_every=6)
    dl.init_fields(0, *(a[:nd, :nd, :nd] for a in (rho, ux, uy, uz)))
    dl.step(6)
    st = dl.subvolume_balance(0, [2, 8, 32])
    torch.cuda.synchronize()
    assert np.all(np.isfinite(st[:, 2:, 0]))
    print("3d case done")


def case_diag(n=512, events=2):
    lat = Lattice([Member(n, n, 0.52)], precision=32, diag_every=200)
    lat.init_fields(0, *li.random_phase(n, seed=1000, u_rms=0.02))
    Ls = li.pow2_sizes(1, 8, n)
    for _ in range(events):
        lat.step(200)
        stats = lat.subvolume_balance(0, Ls)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(stats[:, 2:, 0]))
    print("diag case done:", lat.launch_count, "launches")


def case_diag_batch(members=16, n=512, events=2):
    """One batched diagnostic event over 16 members (Table 1 random boxes),
    as the ensemble benchmark runs it; about 2 GB of device memory."""
    lat = Lattice([Member(n, n, 0.52)] * members, precision=32, diag_every=200)
    for m in range(members):
        lat.init_fields(m, *li.random_phase(n, seed=1000 + m, u_rms=0.02))
    Ls = li.pow2_sizes(1, 8, n)
    origins = [li.table1_origins(n, L, seed=7 + L) for L in Ls]
    for _ in range(events):
        lat.step(200)
        stats = lat.subvolume_balance_batch(range(members), Ls, origins=origins)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(stats[:, :, 2:, 0]))
    print("diag batch case done:", lat.launch_count, "launches")


def case_fp64(n=512, steps=20):
    lat = Lattice([Member(n, n, 0.52)], precision=64)
    lat.init_fields(0, *li.random_phase(n, seed=1000, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("fp64 case done")


def case_adjoint(n=256, steps=6):
    F0 = li.kolmogorov_F0(n, 0.55, 4, 1e-4, 0.03)
    lat = Lattice([Member(n, n, 0.55, 1.0, 1, 4, F0, 1e-4)], precision=64)
    lat.init_fields(0, *li.random_phase(n, seed=0, u_rms=0.02))
    f = lat.get_populations(0)
    lam = torch.zeros_like(f)
    out = torch.empty_like(f)
    acc = torch.zeros(2, dtype=torch.float64, device=f.device)
    for _ in range(steps):
        lat.adjoint_step(0, f, lam, out, 1e-3, (0, 0), 16, acc[0:1], acc[1:2])
        lam, out = out, lam
    torch.cuda.synchronize()
    print("adjoint case done")


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "step"
    {"step": case_step, "step_full": case_step_full, "paper_forcing": case_paper_forcing,
     "collisions": case_collisions, "3d": case_3d,
     "diag": case_diag, "diag_batch": case_diag_batch, "fp64": case_fp64,
     "adjoint": case_adjoint}[which]()
