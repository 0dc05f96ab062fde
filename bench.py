#!/usr/bin/env python
"""Benchmark of the D2Q9 LBGK hot path on GB300.

Workload (one bench step): the decaying 2D turbulence ensemble -- 64 members
of 512^2, tau 0.52, FP32 deviation populations, random-phase initial fields
(seed 1000 + member, u_rms 0.02) -- advanced by one diagnostic period of 200
time steps (the batched stream-collide, one launch per step for all
members, replayed from CUDA graphs), and the diagnostic event: the
moment snapshots of the three last time levels and, for every member, the
sub-volume energy/enstrophy balance (terms, summed-area tables, balancing
errors and their statistics) at L = 2, 4, ..., 256 on the paper's Table 1
random boxes (56000 per member), queued on the library's diagnostic stream
so that it runs while the next period steps.  One event over every periodic
origin (2.1 M boxes per member), and one Table 1 event on its own, are timed
beside it.

Metric: aggregate GLUPS (lattice updates per second over all members and
GPUs, diagnostics included), plus the roofline of the dominant kernel
(stream-collide, 72 algorithmic bytes per update), the plain single-instance
FP64 step beside it, an end-to-end figure through the C ABI with host
buffers, and the FP64 CPU oracle timed on a bounded sample on the host.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
(N > 1 under torch.distributed.run: members are sharded, weak scaling);
python bench.py --case NAME runs one small profiling case (CASES) instead.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbm_inputs as li  # noqa: E402

METRIC = "D2Q9 GLUPS & % HBM roofline, batched FP32 vs plain FP64 at ≤2e-6 err"
BYTES_PER_LU_F32 = 72
BYTES_PER_LU_F64 = 144
FALLBACK_HBM_GBS = 6800.0
PERIOD = 200           # time steps per bench step (one diagnostic period)
PURE_STEPS = PERIOD - 3  # steps before the three snapshot levels


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default=None,
                    help="run one profiling case instead of the benchmark (see CASES)")
    return ap.parse_args()


def member_seed(seed0: int, rank: int, members_per_rank: int, m: int) -> int:
    """Seed of member m on a rank: the ensemble is sharded by member, so each
    rank runs its own disjoint block of seeds (weak scaling)."""
    return seed0 + rank * members_per_rank + m


def max_over_ranks(seconds: float) -> float:
    """Slowest rank's time (the job's time); host-side, over the process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_glups(world_size: int, lu_per_rank_step: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: updates of all ranks over the slowest rank's time."""
    return world_size * lu_per_rank_step * steps / seconds / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    with open(os.path.join(ROOT, "paper_1809_06735_gb300", "csrc", "lbm_step.cu"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the stream-collide kernel from the committed
    ncu summary, valid only while the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "step_f32_vec_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_full_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        smax = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for k, nm in enumerate(names):
                if s[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# CPU (oracle) sample: one member, one full diagnostic period, diagnostic on
# sampled origins.
# ---------------------------------------------------------------------------

def table1_boxes(n, Ls, scale=1.0):
    """The paper's Table 1 random boxes for each size (seed = L); ``scale``
    < 1 keeps only that fraction of each list (bounded CPU samples)."""
    out = []
    for L in Ls:
        o = li.table1_origins(n, L, seed=L)
        out.append(o[:max(1, int(round(o.shape[0] * scale)))])
    return out


def oracle_period_sample(seed: int, n_steps: int = PERIOD, box_fraction: float = 1.0):
    import oracle
    wl = li.decaying_ensemble_workload()
    n, tau = wl["n"], wl["tau"]
    rho, ux, uy = li.random_phase(n, seed=seed, u_rms=wl["u_rms"])
    f = oracle.init(rho, ux, uy)
    boxes = table1_boxes(n, wl["Ls"], box_fraction)
    t0 = time.perf_counter()
    f_a = oracle.run(f, n_steps - 2, tau)
    f_b = oracle.run(f_a, 1, tau)
    f_c = oracle.run(f_b, 1, tau)
    T = oracle.terms_from_populations(f_c, f_b, f_a, tau)
    for L, o in zip(wl["Ls"], boxes):
        oracle.balance_stats(T, [L], origins=o)
    dt = time.perf_counter() - t0
    return n * n * n_steps, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    import oracle
    oracle.build()
    wl = li.decaying_ensemble_workload()
    for w in range(args.warmup):
        oracle_period_sample(wl["seed0"] + w, n_steps=20, box_fraction=0.01)
    lu, secs = 0, 0.0
    for k in range(args.steps):
        a, b = oracle_period_sample(wl["seed0"] + k, n_steps=20, box_fraction=0.01)
        lu += a
        secs += b
    v = lu / secs / 1e9
    sample = ("per step: one 512^2 member of the 64, 20 LBM steps of the 200-step period, "
              "then the diagnostic on 1% of the Table 1 random boxes per L (L=2..256)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def paper_forcing_leg(P, stream, dev, peak):
    """The paper's own turbulence forcing (eqs. 14-16, force kind 2) at its
    grid and amplitudes: 64 FP32 members of 256^2, F^T_0 = 8e-4, phase 0,
    F^R_0 = 1e-5, tau = 0.52.  A step is the damping projection (one read of
    the populations, 36 B/LU) plus the stream-collide with the shell-force
    table (72 + 8 B/LU): 116 algorithmic bytes per lattice update."""
    import torch
    n2, M2, steps = 256, 64, 200
    lat = P.Lattice([P.Member(n2, n2, 0.52, 1.0, 2, 0, 8e-4, 0.0, 0.0, 1e-5)] * M2,
                    precision=32, graph_steps=50, stream=stream, device=dev)
    for m in range(M2):
        lat.init_fields(m, *li.random_phase(n2, seed=3000 + m, u_rms=0.02))
    lat.step(100)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    lat.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    secs = a.elapsed_time(b) / 1e3
    lu = M2 * n2 * n2 * steps
    gbs = 116.0 * lu / secs / 1e9
    tune = lat.tuning()
    del lat
    return {"members": M2, "grid": [n2, n2], "FT0": 8e-4, "FR0": 1e-5, "glups": lu / secs / 1e9,
            "bytes_per_lu": 116, "achieved_gbs": gbs, "frac": gbs / peak,
            "storage": tune["storage"]}


def collision_models_leg(P, stream, dev, peak):
    """The variable-viscosity collisions (Sec. 1) on 16 FP32 members of
    512^2 (tau0 = 0.51): Smagorinsky (Cs = 0.1) and eq. (7) on the extended
    vectorised kernel, the entropic LBM (its per-cell root finding) on the
    general kernel.  Every step moves 72 algorithmic bytes per update."""
    import torch
    n, M, steps = 512, 16, 40
    fields = li.random_phase(n, seed=4000, u_rms=0.02)
    out = {"members": M, "grid": [n, n], "tau0": 0.51}
    for name, coll, cs in (("smagorinsky", 1, 0.1), ("eq7", 2, 0.0), ("elbm", 3, 0.0)):
        lat = P.Lattice([P.Member(n, n, 0.51, collision=coll, Cs=cs)] * M, precision=32,
                        graph_steps=20, stream=stream, device=dev)
        for m in range(M):
            lat.init_fields(m, *fields)
        lat.step(20)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        lat.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        secs = a.elapsed_time(b) / 1e3
        lu = M * n * n * steps
        gbs = BYTES_PER_LU_F32 * lu / secs / 1e9
        out[name] = {"glups": lu / secs / 1e9, "achieved_gbs": gbs, "frac": gbs / peak,
                     "kernel": "k_step_scalar<float>" if coll == 3 else "k_step_f32_vec (extended)",
                     # the entropic collision's per-cell root finding keeps the issue
                     # slots busy (ALU-bound); frac is then only its share of HBM
                     "bound": "alu" if coll == 3 else "hbm"}
        del lat
    return out


def taylor_green_leg(P, stream, dev):
    """The plain FP64 Taylor-Green case: 64^2, tau 0.6, u0 0.01, 1000 steps
    with the balance at L in {4, 8, 16, 32} every 100 steps.  A 64^2 step
    cannot fill the GPU, so its time is launch latency: reported per step
    with plain launches and with graph replay, and for the whole workload
    (steps, snapshots and its ten balance events, host wall clock)."""
    import torch
    wl = li.taylor_green_workload()
    n, tau, D, Ls, steps = wl["n"], wl["tau"], wl["diag_every"], wl["Ls"], wl["steps"]
    rho, ux, uy = li.taylor_green(n, u0=wl["u0"])
    out = {"grid": [n, n], "tau": tau, "steps": steps}
    for key, graph in (("plain", 0), ("graph", 100)):
        lat = P.Lattice([P.Member(n, n, tau)], precision=64, graph_steps=graph, stream=stream,
                        device=dev)
        lat.init_fields(0, rho, ux, uy)
        lat.step(200)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        lat.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        us = a.elapsed_time(b) * 1e3 / steps
        out["us_per_step_" + key] = us
        out["glups_" + key] = n * n / us / 1e3
        lat.close()
    lat = P.Lattice([P.Member(n, n, tau)], precision=64, diag_every=D, graph_steps=16,
                    stream=stream, device=dev)
    lat.init_fields(0, rho, ux, uy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps // D):
        lat.step(D)
        st = lat.subvolume_balance(0, Ls)
    torch.cuda.synchronize()
    out["workload_ms"] = (time.perf_counter() - t0) * 1e3
    out["balance_events"] = steps // D
    assert np.all(np.isfinite(st[:, 2:, 0]))
    lat.close()
    return out


def three_d_leg(P, stream, dev, peak):
    """The three-dimensional extension: 2 FP32 members of 128^3 on D3Q19
    (152 algorithmic bytes per update: 19 populations read and written) and
    on D3Q27 (216 B), and one balance event (all 64^3 periodic origins,
    L = 2..64) on a 64^3 member, FP64 and FP32 term arithmetic."""
    import torch
    n, M, steps = 128, 2, 40
    g = np.random.default_rng(5)
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ux = 0.02 * np.sin(X + 0.3) * np.cos(Y) * np.cos(Z)
    uy = -0.02 * np.cos(X + 0.3) * np.sin(Y) * np.cos(Z) + 0.005 * g.normal() * np.sin(Z)
    uz = 0.005 * np.sin(X - Y)
    rho = np.ones((n, n, n))

    def timed(q):
        lat = P.Lattice3D([P.Member3(n, n, n, 0.52)] * M, precision=32, stream=stream, device=dev,
                          lattice=q)
        for m in range(M):
            lat.init_fields(m, rho, ux, uy, uz)
        lat.step(10)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        lat.step(steps)
        b.record(stream)
        torch.cuda.synchronize()
        secs = a.elapsed_time(b) / 1e3
        lu = M * n ** 3 * steps
        del lat
        return lu / secs / 1e9, 8.0 * q * lu / secs / 1e9

    glups, gbs = timed(19)
    glups27, gbs27 = timed(27)
    nd = 64
    sl = (slice(None, None, 2),) * 3

    def diag_event(precision, diag_precision):
        dl = P.Lattice3D([P.Member3(nd, nd, nd, 0.52)], precision=precision, diag_every=20,
                         stream=stream, device=dev, diag_precision=diag_precision)
        dl.init_fields(0, rho[sl], ux[sl], uy[sl], uz[sl])
        dl.step(20)
        dl.subvolume_balance(0, [2, 4, 8, 16, 32, 64])  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = dl.subvolume_balance(0, [2, 4, 8, 16, 32, 64])
        secs = time.perf_counter() - t0
        assert np.all(np.isfinite(st[:, 2:, 0]))
        del dl
        return secs

    diag_s = diag_event(64, 64)
    diag32_s = diag_event(32, 32)
    return {"members": M, "grid": [n, n, n], "precision": "fp32", "glups": glups,
            "bytes_per_lu": 152, "achieved_gbs": gbs, "frac": gbs / peak,
            "d3q27": {"glups": glups27, "bytes_per_lu": 216, "achieved_gbs": gbs27,
                      "frac": gbs27 / peak},
            "diagnostic_event_ms_fp64_64cubed_all_origins": 1e3 * diag_s,
            "diagnostic_event_ms_fp32_64cubed_all_origins": 1e3 * diag32_s}


def workload_config():
    wl = li.decaying_ensemble_workload()
    return {"workload": wl["name"], "members_per_gpu": wl["members"], "grid": [wl["n"], wl["n"]],
            "tau": wl["tau"], "precision": "fp32 deviation populations; diagnostic terms in fp32 from compensated snapshots, exact int64 box sums, fp64 statistics",
            "lbm_steps_per_step": PERIOD,
            "diagnostic": "per step, every member: balance terms + SAT + the paper's "
                          "Table 1 random boxes (56000 per member) at L=2..256",
            "l2": "inputs larger than L2 (1.2 GB of populations per GPU), no flush"}


# ---------------------------------------------------------------------------
# Profiling cases (python bench.py --case NAME): small, self-contained runs of
# each kernel family for Nsight Compute.  Sizes keep the working set above the
# L2 (so DRAM counters mean something) and below a few GB.  The step cases
# create their handle with the launch-shape autotuner on: 2 storages x 18
# shapes x 8 launches = 288 launches of k_step_f32_vec come before the first
# step of the run.
# ---------------------------------------------------------------------------


def case_step(P, members=16, n=512, steps=25):
    import torch
    lat = P.Lattice([P.Member(n, n, 0.52)] * members, precision=32, graph_steps=0)
    for m in range(members):
        lat.init_fields(m, *li.random_phase(n, seed=1000 + m, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("step case done:", lat.launch_count, "launches")


def case_step_full(P, members=64, n=512, steps=200):
    """The ensemble benchmark's stream-collide workload (64 x 512^2, FP32,
    autotuned storage and shape) for single-pass DRAM counters; the
    autotuner's 288 launches and the 64 initialisations come first."""
    import torch
    lat = P.Lattice([P.Member(n, n, 0.52)] * members, precision=32, graph_steps=0, diag_batch=1)
    for m in range(members):
        lat.init_fields(m, *li.random_phase(n, seed=1000 + m, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("step_full case done:", lat.launch_count, "launches", lat.tuning())


def case_paper_forcing(P, members=64, n=256, steps=30):
    """The paper's forcing (force kind 2) on 64 FP32 members of 256^2: the
    damping projection and the stream-collide with the shell-force table."""
    import torch
    lat = P.Lattice([P.Member(n, n, 0.52, 1.0, 2, 0, 8e-4, 0.0, 0.0, 1e-5)] * members,
                  precision=32, graph_steps=0)
    for m in range(members):
        lat.init_fields(m, *li.random_phase(n, seed=3000 + m, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("paper forcing case done:", lat.launch_count, "launches", lat.tuning())


def case_collisions(P, members=16, n=512, steps=12):
    """The variable-viscosity collisions on 16 FP32 members of 512^2: one
    handle each for Smagorinsky, eq. (7) and the entropic LBM."""
    import torch
    fields = li.random_phase(n, seed=4000, u_rms=0.02)
    for coll, cs in ((1, 0.1), (2, 0.0), (3, 0.0)):
        lat = P.Lattice([P.Member(n, n, 0.51, collision=coll, Cs=cs)] * members, precision=32,
                      graph_steps=0)
        for m in range(members):
            lat.init_fields(m, *fields)
        lat.step(steps)
        torch.cuda.synchronize()
        print("collision", coll, "done:", lat.launch_count, "launches", lat.tuning())
        del lat


def case_3d(P, members=2, n=128, steps=12):
    """The D3Q19 and D3Q27 stream-collide on 2 FP32 members of 128^3 each,
    then one FP64 balance event on a 48^3 member."""
    import torch
    x = 2 * np.pi * np.arange(n) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ux, uy = 0.02 * np.sin(X) * np.cos(Y) * np.cos(Z), -0.02 * np.cos(X) * np.sin(Y) * np.cos(Z)
    uz, rho = 0.005 * np.sin(X - Y), np.ones((n, n, n))
    for q in (19, 27):
        lat = P.Lattice3D([P.Member3(n, n, n, 0.52)] * members, precision=32, lattice=q)
        for m in range(members):
            lat.init_fields(m, rho, ux, uy, uz)
        lat.step(steps)
        torch.cuda.synchronize()
        del lat
    nd = 48
    dl = P.Lattice3D([P.Member3(nd, nd, nd, 0.52)], precision=64, diag_every=6)
    dl.init_fields(0, *(a[:nd, :nd, :nd] for a in (rho, ux, uy, uz)))
    dl.step(6)
    st = dl.subvolume_balance(0, [2, 8, 32])
    torch.cuda.synchronize()
    assert np.all(np.isfinite(st[:, 2:, 0]))
    print("3d case done")


def case_diag(P, n=512, events=2):
    import torch
    lat = P.Lattice([P.Member(n, n, 0.52)], precision=32, diag_every=200)
    lat.init_fields(0, *li.random_phase(n, seed=1000, u_rms=0.02))
    Ls = li.pow2_sizes(1, 8, n)
    for _ in range(events):
        lat.step(200)
        stats = lat.subvolume_balance(0, Ls)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(stats[:, 2:, 0]))
    print("diag case done:", lat.launch_count, "launches")


def case_diag_batch(P, members=16, n=512, events=2):
    """One batched diagnostic event over 16 members (Table 1 random boxes),
    as the ensemble benchmark runs it; about 2 GB of device memory."""
    import torch
    lat = P.Lattice([P.Member(n, n, 0.52)] * members, precision=32, diag_every=200)
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


def case_fp64(P, n=512, steps=20):
    import torch
    lat = P.Lattice([P.Member(n, n, 0.52)], precision=64)
    lat.init_fields(0, *li.random_phase(n, seed=1000, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("fp64 case done")


def case_adjoint(P, n=256, steps=6):
    import torch
    F0 = li.kolmogorov_F0(n, 0.55, 4, 1e-4, 0.03)
    lat = P.Lattice([P.Member(n, n, 0.55, 1.0, 1, 4, F0, 1e-4)], precision=64)
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


CASES = {name[5:]: fn for name, fn in list(globals().items()) if name.startswith("case_")}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1809_06735_gb300 as P
    P.load_library()

    wl = li.decaying_ensemble_workload()
    n, tau, M = wl["n"], wl["tau"], wl["members"]
    stream = torch.cuda.current_stream(dev)
    lat = P.Lattice([P.Member(n, n, tau)] * M, precision=32, diag_every=PERIOD,
                    graph_steps=PURE_STEPS - 1, stream=stream, device=dev)
    # pinned host initial fields [rho, ux, uy][member][y][x] (also the e2e inputs)
    host = torch.empty((3, M, n, n), dtype=torch.float64, pin_memory=True)
    for m in range(M):
        r, u, v = li.random_phase(n, seed=member_seed(wl["seed0"], rank, M, m), u_rms=wl["u_rms"])
        host[0, m].copy_(torch.from_numpy(r))
        host[1, m].copy_(torch.from_numpy(u))
        host[2, m].copy_(torch.from_numpy(v))
    hnp = host.numpy()
    dev_fields = host.to(dev)
    for m in range(M):
        lat.init_fields(m, dev_fields[0, m], dev_fields[1, m], dev_fields[2, m])
    torch.cuda.synchronize()
    Ls = wl["Ls"]
    all_members = list(range(M))
    boxes = table1_boxes(n, Ls)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    stats_buf = [torch.empty((M, len(Ls), 15, 2), dtype=torch.float64, device=dev)
                 for _ in range(2)]

    def bench_step(k, rec=None):
        # the diagnostic of this period runs on the library's diagnostic
        # stream while the next period's stream-collide proceeds
        if rec is not None:
            rec[0].record(stream)
        lat.step(PURE_STEPS)
        if rec is not None:
            rec[1].record(stream)
        lat.step(PERIOD - PURE_STEPS)
        return lat.subvolume_balance_async(all_members, Ls, origins=boxes,
                                           out=stats_buf[k % 2])

    for w in range(args.warmup):
        bench_step(w)
    lat.diag_synchronize()
    torch.cuda.synchronize()
    recs = [(ev(), ev()) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    # no cyclic garbage collection inside a timed region: a handle destroyed
    # there (its graphs and streams) would stall the queued work
    gc.collect()
    gc.disable()
    clocks.start()
    launches0 = lat.launch_count
    t0, t1 = ev(), ev()
    t0.record(stream)
    stats = None
    for k in range(args.steps):
        stats = bench_step(k, recs[k])
    lat.diag_synchronize()  # the last period's diagnostic is part of the job
    t1.record(stream)
    torch.cuda.synchronize()
    gc.enable()
    stats = stats.cpu().numpy()
    clk = clocks.stop()
    launches = lat.launch_count - launches0
    elapsed = t0.elapsed_time(t1) / 1e3
    pure = sum(a.elapsed_time(b) for a, b in recs) / 1e3
    if ws > 1:
        elapsed = max_over_ranks(elapsed)
    assert stats is not None and np.all(np.isfinite(stats[:, :, 2:, 0]))
    lu_per_gpu_step = M * n * n * PERIOD
    value = aggregate_glups(ws, lu_per_gpu_step, args.steps, elapsed)
    kern_s = pure / (args.steps * PURE_STEPS)
    step_glups = M * n * n / kern_s / 1e9
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_LU_F32 * M * n * n / kern_s / 1e9

    # one diagnostic event of all members on its own: the Table 1 boxes of the
    # timed steps, and every periodic origin (2.1 M boxes per member)
    diag_ms = {}
    for key, org in (("table1_boxes", boxes), ("all_origins", None)):
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record(stream)
        st = lat.subvolume_balance_batch(all_members, Ls, origins=org)
        b.record(stream)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(st[:, :, 2:, 0]))
        diag_ms[key] = a.elapsed_time(b)

    # plain single-instance FP64 step on one 512^2 member
    lat64 = P.Lattice([P.Member(n, n, tau)], precision=64, graph_steps=20, stream=stream,
                      device=dev)
    lat64.init_fields(0, dev_fields[0, 0], dev_fields[1, 0], dev_fields[2, 0])
    lat64.step(40)
    a, b = ev(), ev()
    torch.cuda.synchronize()
    a.record(stream)
    lat64.step(200)
    b.record(stream)
    torch.cuda.synchronize()
    fp64_s = a.elapsed_time(b) / 1e3 / 200
    fp64_glups = n * n / fp64_s / 1e9
    del lat64
    paper_forcing = paper_forcing_leg(P, stream, dev, measured_peaks()[0])
    collisions = collision_models_leg(P, stream, dev, measured_peaks()[0])
    three_d = three_d_leg(P, stream, dev, measured_peaks()[0])
    taylor_green = taylor_green_leg(P, stream, dev)

    # end to end through the public API with host buffers: every step uploads
    # the initial fields of all members from pinned host memory, runs the
    # period and reads its statistics back to the host.  Pipelined as a
    # production caller would: step k's upload (copy stream) and step k-1's
    # statistics read overlap step k's stream-collide; the diagnostic runs
    # on the library's diagnostic stream.
    e2e_steps = max(1, args.steps)
    dev_in = torch.empty((3, M, n, n), dtype=torch.float64, device=dev)
    copy_stream = torch.cuda.Stream(device=dev)
    copied, consumed = torch.cuda.Event(), torch.cuda.Event()
    host_stats = torch.empty((e2e_steps + 1, M, len(Ls), 15, 2), dtype=torch.float64,
                             pin_memory=True)
    e2e_buf = [torch.empty((M, len(Ls), 15, 2), dtype=torch.float64, device=dev)
               for _ in range(2)]

    up0, up1 = ev(), ev()  # the first upload: the pipeline fill, not hidden

    def e2e_run(nsteps, record):
        for k in range(nsteps):
            copy_stream.wait_event(consumed)  # the previous step's init has read dev_in
            if k == 0:
                up0.record(copy_stream)
            with torch.cuda.stream(copy_stream):
                dev_in.copy_(host, non_blocking=True)
            copied.record(copy_stream)
            if k == 0:
                up1.record(copy_stream)
            stream.wait_event(copied)
            lat.init_fields_batch(all_members, dev_in[0], dev_in[1], dev_in[2])
            consumed.record(stream)
            lat.step(PERIOD)
            if k > 0:  # step k-1's statistics to the host while step k runs
                lat.diag_synchronize()
                with torch.cuda.stream(copy_stream):
                    record[k - 1].copy_(e2e_buf[(k - 1) % 2], non_blocking=True)
            if k > 1:  # the read of step k-2's statistics has left e2e_buf[k % 2]
                copy_stream.synchronize()
            lat.subvolume_balance_async(all_members, Ls, origins=boxes, out=e2e_buf[k % 2])
        lat.diag_synchronize()
        with torch.cuda.stream(copy_stream):
            record[nsteps - 1].copy_(e2e_buf[(nsteps - 1) % 2], non_blocking=True)
        copy_stream.synchronize()

    e2e_run(1, host_stats)  # warm-up: the step graph of the storage parity after a restart
    runs, uploads = [], []
    gc.collect()
    gc.disable()  # as in the timed steps above
    for _ in range(3):  # median of three pipelined runs: host-side jitter is one-sided
        torch.cuda.synchronize()
        te = time.perf_counter()
        e2e_run(e2e_steps, host_stats)
        torch.cuda.synchronize()
        runs.append(time.perf_counter() - te)
        uploads.append(up0.elapsed_time(up1))
    gc.enable()
    assert np.all(np.isfinite(host_stats[:e2e_steps, :, :, 2:, 0].numpy()))
    te = float(np.median(runs))
    if ws > 1:
        te = max_over_ranks(te)
    e2e = {"value": ws * lu_per_gpu_step * e2e_steps / te / 1e9, "unit": "GLUPS",
           "h2d_bytes_per_step": int(M * 3 * n * n * 8),
           "d2h_bytes_per_step": int(M * len(Ls) * 30 * 8),
           "note": "per step: pinned host fields of all members uploaded (copy stream) and "
                   "initialised through lbm_init_fields_batch, 200 steps, Table 1 statistics "
                   "to pinned host memory; step k's upload and step k-1's statistics "
                   "overlap step k; wall clock over %d steps including pipeline fill and "
                   "drain, median of 3 runs (%s ms; the first upload, not overlapped: %s ms)"
                   % (e2e_steps, ", ".join("%.1f" % (1e3 * r) for r in runs),
                      ", ".join("%.1f" % u for u in uploads))}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        lu, secs = oracle_period_sample(wl["seed0"])
        cpu = {"value": lu / secs / 1e9, "unit": "GLUPS", "cores": 1, "kind": "oracle",
               "sample": "one 512^2 member of the 64: the full 200-step period, then the "
                         "diagnostic on the same Table 1 random boxes (L=2..256)",
               "seconds": secs}

    if rank == 0:
        traffic = profiled_traffic()
        line = {
            "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(),
            "roofline": {"bound": "hbm", "kernel": "k_step_f32_vec", "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": BYTES_PER_LU_F32 * M * n * n,
                         "avg_launch_ms": kern_s * 1e3},
            "step_only_glups_per_gpu": step_glups,
            "diagnostic_event_ms": dict(diag_ms, members=M, sizes=list(Ls)),
            "fp64_plain_single_instance": {"glups": fp64_glups, "grid": [n, n],
                                           "ratio_batched_fp32_over_fp64": step_glups / fp64_glups},
            "paper_forcing_ensemble": paper_forcing,
            "collision_models": collisions,
            "three_d": three_d,
            "fp64_taylor_green_64": taylor_green,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def main():
    args = parse()
    if args.case is not None:
        import paper_1809_06735_gb300 as P
        P.load_library()
        CASES[args.case](P)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
