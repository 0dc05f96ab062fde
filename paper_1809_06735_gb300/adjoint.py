"""Reverse-mode gradients of a time-averaged sub-volume balance quantity.

Objective (the differentiation workload):
    J(tau, F0, f0) = 1/(n1 - n0 + 1) * sum_{n = n0}^{n1} <RHS^{E,4}>_V (n),
the L x L box average (origin ``box``) of the dissipation term of eq. (8),
evaluated on the states f(n) of the forced D2Q9 LBGK model of eq. (1) started
from f0, with relaxation time tau and Kolmogorov amplitude F0.

Forward: the batched CUDA step, with a checkpoint of the public state every
``checkpoint_every`` steps (device memory).  Backward: for each checkpoint
interval, from the last to the first, the states are recomputed from the
checkpoint and the adjoint step kernel (transposed streaming + transposed
BGK/EDM Jacobian + the objective's own adjoint) is applied step by step,
accumulating dJ/dtau and dJ/dF0 in FP64 on the device.  The adjoint
arithmetic is FP64 whatever the forward precision.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import Lattice, Member


@dataclass
class ObjectiveSpec:
    nx: int
    ny: int
    kf: int
    alpha: float
    n0: int
    n1: int
    box: tuple
    L: int
    precision: int = 64
    checkpoint_every: int = 100
    rho0: float = 1.0


def _lattice(spec: ObjectiveSpec, tau: float, F0: float) -> Lattice:
    m = Member(spec.nx, spec.ny, float(tau), spec.rho0, 1, spec.kf, float(F0), spec.alpha)
    return Lattice([m], precision=spec.precision)


def forward_objective(spec: ObjectiveSpec, tau: float, F0: float, f0: torch.Tensor,
                      keep_checkpoints: bool = False):
    """Run the model from f0 (public FP64 populations, device) and return
    J (device FP64 scalar tensor) and, optionally, the checkpoints."""
    lat = _lattice(spec, tau, F0)
    lat.set_populations(0, f0)
    w = 1.0 / (spec.n1 - spec.n0 + 1)
    acc = torch.zeros(1, dtype=torch.float64, device=f0.device)
    ckpts = {}
    K = spec.checkpoint_every
    n = 0
    while True:
        if keep_checkpoints and n % K == 0:
            ckpts[n] = lat.get_populations(0).clone()
        if n == spec.n1:
            lat.objective_accumulate(0, w, spec.box, spec.L, acc)
            break
        target = min((n // K + 1) * K, spec.n1)
        if n < spec.n0:  # no objective term before n0
            target = min(target, spec.n0)
            lat.step(target - n)
        else:  # objective at n .. target - 1, stepping to target
            lat.objective_steps(0, target - n, w, spec.box, spec.L, acc)
        n = target
    return acc[0], ckpts, lat


def adjoint_objective(spec: ObjectiveSpec, tau: float, F0: float, lat: Lattice, ckpts: dict):
    """Gradients (dJ/dtau, dJ/dF0, dJ/df0) by checkpointed reverse sweeps:
    each interval is recomputed from its checkpoint into a device buffer of
    states, then swept backwards in one library call."""
    dev = next(iter(ckpts.values())).device
    w = 1.0 / (spec.n1 - spec.n0 + 1)
    shape = (9, spec.ny, spec.nx)
    lam_a = torch.empty(shape, dtype=torch.float64, device=dev)
    lam_b = torch.empty_like(lam_a)
    lam_tmp = torch.empty_like(lam_a)
    dtau = torch.zeros(1, dtype=torch.float64, device=dev)
    dF0 = torch.zeros(1, dtype=torch.float64, device=dev)
    K = spec.checkpoint_every
    states = torch.empty((K,) + shape, dtype=torch.float64, device=dev)
    lam_in, lam_out = None, lam_a
    for c in sorted(ckpts, reverse=True):
        hi = min(c + K - 1, spec.n1)
        ns = hi - c + 1
        lat.set_populations(0, ckpts[c])
        lat.record_trajectory(0, states[:ns])
        weights = [w if c + k >= spec.n0 else 0.0 for k in range(ns)]
        lat.adjoint_sweep(0, states[:ns], lam_in, lam_out, lam_tmp, weights, spec.box, spec.L,
                          dtau, dF0)
        lam_in, lam_out = lam_out, (lam_b if lam_out is lam_a else lam_a)
    return dtau[0], dF0[0], lam_in


class BoxDissipation(torch.autograd.Function):
    """J(tau, F0, f0) with gradients from the hand-written adjoint kernels.

    tau, F0: 0-dim float64 tensors; f0: [9, ny, nx] float64 device tensor of
    public pre-collision populations."""

    @staticmethod
    def forward(ctx, tau, F0, f0, spec: ObjectiveSpec):
        t, a = float(tau), float(F0)
        J, ckpts, lat = forward_objective(spec, t, a, f0.detach().contiguous(),
                                          keep_checkpoints=True)
        ctx.spec, ctx.t, ctx.a, ctx.ckpts, ctx.lat = spec, t, a, ckpts, lat
        return J.clone()

    @staticmethod
    def backward(ctx, gJ):
        dtau, dF0, lam0 = adjoint_objective(ctx.spec, ctx.t, ctx.a, ctx.lat, ctx.ckpts)
        ctx.lat.close()
        g = gJ.to(torch.float64)
        return (g * dtau).reshape(()), (g * dF0).reshape(()), g * lam0, None


def box_dissipation(tau, F0, f0, spec: ObjectiveSpec):
    return BoxDissipation.apply(tau, F0, f0, spec)
