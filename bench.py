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
    """One member of the decaying ensemble through the oracle: n_steps LBM
    steps, then the diagnostic of the last three levels on the Table 1
    boxes (a fraction of them).  Returns (updates, step seconds, diagnostic
    seconds)."""
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
    t1 = time.perf_counter()
    T = oracle.terms_from_populations(f_c, f_b, f_a, tau)
    for L, o in zip(wl["Ls"], boxes):
        oracle.balance_stats(T, [L], origins=o)
    t2 = time.perf_counter()
    return n * n * n_steps, t1 - t0, t2 - t1


def _oracle_member_task(args):
    """Pool task (spawned process): one member's oracle period sample."""
    return oracle_period_sample(*args)


def _oracle_strip_task(args):
    """Pool task: `steps` oracle steps of one 8192 x (rows + 2 steps) strip
    of the large forced run (random near-rest populations: the oracle's
    cost does not depend on the values), as a window of the 8192^2 grid
    (exact in its interior).  Returns (interior updates, seconds)."""
    import oracle
    y0, rows, steps = args
    wl = li.large_forced_workload()
    n = wl["n"]
    f = li.random_populations(n, rows + 2 * steps, seed=y0)
    force = oracle.Force(1, wl["F0"], wl["kf"], wl["alpha"])
    t0 = time.perf_counter()
    oracle.run_window(f, steps, wl["tau"], force, 0, y0 - steps, n, n)
    return n * rows * steps, time.perf_counter() - t0


def _oracle_taylor_green_task(_):
    """Pool task: the whole 64^2 FP64 Taylor-Green workload through the
    oracle (1000 steps, the balance at L in {4, 8, 16, 32} over every
    periodic origin every 100 steps).  Returns seconds."""
    import oracle
    wl = li.taylor_green_workload()
    n, tau, D = wl["n"], wl["tau"], wl["diag_every"]
    f = oracle.init(*li.taylor_green(n, u0=wl["u0"]))
    t0 = time.perf_counter()
    for _ in range(wl["steps"] // D):
        f2 = oracle.run(f, D - 2, tau)
        f1 = oracle.run(f2, 1, tau)
        f = oracle.run(f1, 1, tau)
        oracle.balance_stats(oracle.terms_from_populations(f, f1, f2, tau), wl["Ls"])
    return time.perf_counter() - t0


def oracle_pool(cores: int):
    """A pool of spawned processes for the oracle (no fork after CUDA use)."""
    import multiprocessing as mp
    import oracle
    oracle.build()  # compiled once, before the workers load it
    return mp.get_context("spawn").Pool(cores)


def cpu_baseline_all_cores():
    """The FP64 oracle on every host core, one member per process (the
    ensemble shards by member with nothing shared): one full 200-step period
    of the decaying ensemble's 512^2 members, each followed by its Table 1
    diagnostic; then 2 steps of the 8192^2 large-run shape as one strip per
    core, and the whole 64^2 Taylor-Green workload on one core."""
    cores = os.cpu_count() or 1
    wl = li.decaying_ensemble_workload()
    with oracle_pool(cores) as pool:
        pool.map(abs, range(cores))  # workers up (interpreter start, imports)
        t0 = time.perf_counter()
        res = pool.map(_oracle_member_task, [(wl["seed0"] + m, PERIOD, 1.0) for m in range(cores)])
        wall = time.perf_counter() - t0
        rows = 8192 // cores
        t1 = time.perf_counter()
        strips = pool.map(_oracle_strip_task, [(k * rows, rows, 2) for k in range(cores)])
        wall4 = time.perf_counter() - t1
        tg = pool.map(_oracle_taylor_green_task, [0])[0]
    lu = sum(r[0] for r in res)
    step_s = [r[1] for r in res]
    return {"value": lu / wall / 1e9, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": "%d members of 512^2 (one per core, processes): the full 200-step "
                      "period, then the Table 1 diagnostic (L=2..256); GLUPS over the "
                      "wall clock including the diagnostic" % cores,
            "seconds": wall,
            "single_core_step_glups": float(np.median([PERIOD * 512 * 512 / t
                                                        for t in step_s])) / 1e9,
            "diagnostic_s_per_event_512sq_member": float(np.median([r[2] for r in res])),
            "large_8192sq_shape": {"glups": sum(r[0] for r in strips) / wall4 / 1e9,
                                   "cores": cores,
                                   "sample": "2 steps of 8192^2 as %d strips of 8192 x %d "
                                             "(window runs)" % (cores, rows)},
            "taylor_green_64_workload_s": tg}


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    wl = li.decaying_ensemble_workload()
    cores = os.cpu_count() or 1
    with oracle_pool(cores) as pool:
        pool.map(abs, range(cores))

        def one_step(k):
            tasks = [(wl["seed0"] + k * cores + m, 20, 0.01) for m in range(cores)]
            t0 = time.perf_counter()
            res = pool.map(_oracle_member_task, tasks)
            return sum(r[0] for r in res), time.perf_counter() - t0

        for w in range(args.warmup):
            one_step(w)
        lu, secs = 0, 0.0
        for k in range(args.steps):
            a, b = one_step(k)
            lu += a
            secs += b
    v = lu / secs / 1e9
    sample = ("per step: %d of the 512^2 members at once, one per host core (processes), "
              "each 20 LBM steps of the 200-step period, then the diagnostic on 1%% of the "
              "Table 1 random boxes per L (L=2..256)" % cores)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def median_timed(stream, fn, runs=5):
    """Median over `runs` calls of fn() of its device time on `stream`
    (CUDA events, synchronised on both sides), seconds."""
    import torch
    times = []
    for _ in range(runs):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
    return float(np.median(times))


def paper_forcing_leg(P, stream, dev, peak):
    """The paper's own turbulence forcing (eqs. 14-16, force kind 2) at its
    grid and amplitudes: 64 FP32 members of 256^2, F^T_0 = 8e-4, phase 0,
    F^R_0 = 1e-5, tau = 0.52.  At these amplitudes the flow leaves the
    low-Mach range within about 250 steps of a u_rms = 0.02 start and then
    diverges (the FP64 oracle does the same), so every timed run starts
    from the initial fields again: re-initialisation, 10 untimed steps, 100
    timed steps (about 0.05 u_rms at the end), median of five; all members
    are checked finite afterwards.  A step is the damping projection (one
    read of the populations, 36 B/LU) plus the stream-collide with the
    shell-force table (72 + 8 B/LU): 116 algorithmic bytes per update."""
    n2, M2, steps = 256, 64, 100
    lat = P.Lattice([P.Member(n2, n2, 0.52, 1.0, 2, 0, 8e-4, 0.0, 0.0, 1e-5)] * M2,
                    precision=32, graph_steps=50, stream=stream, device=dev)
    fields = [li.random_phase(n2, seed=3000 + m, u_rms=0.02) for m in range(M2)]
    stacked = [np.stack([f[q] for f in fields]) for q in range(3)]
    times = []
    for _ in range(5):
        lat.init_fields_batch(list(range(M2)), *stacked)
        lat.step(10)
        times.append(median_timed(stream, lambda: lat.step(steps), runs=1))
    secs = float(np.median(times))
    finite = all(lat.member_status(m) == 0 for m in range(M2))
    lu = M2 * n2 * n2 * steps
    tune = lat.tuning()
    gbs = 116.0 * lu / secs / 1e9
    del lat
    return {"members": M2, "grid": [n2, n2], "FT0": 8e-4, "FR0": 1e-5, "glups": lu / secs / 1e9,
            "bytes_per_lu": 116, "achieved_gbs": gbs, "frac": gbs / peak,
            "steps_per_run": steps, "fresh_state_runs": True, "finite": finite,
            "storage": tune["storage"], "projection_rows": tune["projection_rows"],
            "kernels_per_step": tune["kernels_per_step"]}


# The forced tau-sweep of the paper's Sec. 5 under its own forcing (eqs.
# 14-16) at amplitudes for which every tau of the sweep reaches a
# statistically stationary low-Mach state on 256^2 (the printed
# F^T_0 = 8e-4, F^R_0 = 1e-5 diverge within about 250 steps under the reading
# of the forcing used here).
TREND_TAUS = (0.6, 0.54, 0.53, 0.52, 0.515)
TREND_FT0, TREND_FR0 = 2e-5, 1e-2
TREND_LS = (2, 3, 4, 8, 16, 32, 64, 128, 181, 256)


def forced_tau_trend(P, members=4, n=256, spin=8000, every=400, events=25, stream=None,
                     dev=None):
    """Balancing-error statistics of the forced sweep: for each tau, `members`
    members of n^2 from random-phase starts (u_rms 0.01, seeds 6000 + m), `spin`
    steps to the stationary state, then `events` balance events `every` steps
    apart (the paper samples 25 configurations in time) over all periodic
    origins at the sizes TREND_LS (L = 3 is l ~ 0.01 and L = 181 l ~ 0.707 on
    256^2).  Returns {tau: {"urms", "finite", "dE"/"dZ": [nL][mean, std]}},
    the statistics averaged over members and events."""
    out = {}
    for tau in TREND_TAUS:
        kw = {} if stream is None else {"stream": stream, "device": dev}
        lat = P.Lattice([P.Member(n, n, tau, 1.0, 2, 0, TREND_FT0, 0.0, 0.0, TREND_FR0)] * members,
                        precision=32, graph_steps=100, diag_every=every, **kw)
        for m in range(members):
            lat.init_fields(m, *li.random_phase(n, seed=6000 + m, u_rms=0.01))
        lat.step(spin)
        acc, urms = [], []
        for _ in range(events):
            lat.step(every)
            acc.append(np.asarray(lat.subvolume_balance_batch(range(members), list(TREND_LS)))[:, :, :2, :])
            urms.append(float(np.sqrt(2 * lat.global_balance(0)[3])))
        a = np.mean(np.stack(acc), axis=(0, 1))  # [nL, quantity, (mean, std)]
        out[tau] = {"urms": float(np.mean(urms)),
                    "finite": all(lat.member_status(m) == 0 for m in range(members)),
                    "dE": a[:, 0, :].tolist(), "dZ": a[:, 1, :].tolist()}
        del lat
    return out


def forced_tau_trend_leg(P, stream, dev):
    """The forced tau-sweep trend (Sec. 5): per tau the mean and std of the
    energy and enstrophy balancing errors at l ~ 0.01 (L = 3) and l ~ 0.707
    (L = 181) of 256^2, and the wall time of the whole sweep."""
    t0 = time.perf_counter()
    res = forced_tau_trend(P, stream=stream, dev=dev)
    i_s, i_l = TREND_LS.index(3), TREND_LS.index(181)
    rows = {}
    for tau, r in res.items():
        rows[str(tau)] = {"urms": round(r["urms"], 4), "finite": r["finite"],
                          "dE_small": r["dE"][i_s], "dE_large": r["dE"][i_l],
                          "dZ_small": r["dZ"][i_s], "dZ_large": r["dZ"][i_l]}
    return {"grid": [256, 256], "members": 4, "FT0": TREND_FT0, "FR0": TREND_FR0,
            "taus": list(TREND_TAUS), "events": 25, "event_every": 400, "spin_up": 8000,
            "stats": "[mean, std] of delta over all periodic origins, averaged over members "
                     "and events", "per_tau": rows,
            "wall_s": time.perf_counter() - t0}


def collision_models_leg(P, stream, dev, peak):
    """The variable-viscosity collisions (Sec. 1) on 16 FP32 members of
    512^2 (tau0 = 0.51): Smagorinsky (Cs = 0.1), eq. (7) and the entropic
    LBM (its per-cell root of the entropy condition) on the vectorised
    kernel.  Every step moves 72 algorithmic bytes per update.  Median of
    five timed 40-step runs."""
    n, M, steps = 512, 16, 40
    fields = li.random_phase(n, seed=4000, u_rms=0.02)
    out = {"members": M, "grid": [n, n], "tau0": 0.51}
    for name, coll, cs in (("smagorinsky", 1, 0.1), ("eq7", 2, 0.0), ("elbm", 3, 0.0)):
        lat = P.Lattice([P.Member(n, n, 0.51, collision=coll, Cs=cs)] * M, precision=32,
                        graph_steps=20, stream=stream, device=dev)
        for m in range(M):
            lat.init_fields(m, *fields)
        lat.step(20)
        secs = median_timed(stream, lambda: lat.step(steps))
        lu = M * n * n * steps
        gbs = BYTES_PER_LU_F32 * lu / secs / 1e9
        out[name] = {"glups": lu / secs / 1e9, "achieved_gbs": gbs, "frac": gbs / peak,
                     "kernel": "k_step_f32_vec (entropic)" if coll == 3 else "k_step_f32_vec (extended)",
                     "bound": "hbm"}
        if coll == 3:  # the entropic root keeps the issue slots busy: ALU-bound
            out[name].update({"bound": "alu", "hbm_frac": gbs / peak})
            wi = issue_counts().get("k_step_f32_vec (entropic)")
            if wi is not None:
                rate = wi * lu / secs
                pk = issue_peak(dev.index or 0)
                out[name].update({"warp_instr_per_lu": wi, "achieved": rate / 1e12,
                                  "peak": pk / 1e12, "unit": "T warp instr/s",
                                  "frac": rate / pk})
        del lat
    return out


def taylor_green_leg(P, stream, dev):
    """The plain FP64 Taylor-Green case: 64^2, tau 0.6, u0 0.01, 1000 steps
    with the balance at L in {4, 8, 16, 32} every 100 steps.  A 64^2 step
    cannot fill the GPU, so its time is latency: reported per step with all
    the steps of a call in one cooperative launch (grid barrier between
    steps; graph_steps = 0) and with graph replay of per-step launches, the
    cost of one grid barrier alone, and the whole workload (steps,
    snapshots and its ten balance events, host wall clock)."""
    import torch
    wl = li.taylor_green_workload()
    n, tau, D, Ls, steps = wl["n"], wl["tau"], wl["diag_every"], wl["Ls"], wl["steps"]
    rho, ux, uy = li.taylor_green(n, u0=wl["u0"])
    out = {"grid": [n, n], "tau": tau, "steps": steps}
    for key, graph in (("cooperative", 0), ("graph", 100)):
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
    P.probe_grid_barrier(128, 1000, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.probe_grid_barrier(128, 20000, stream=stream)
    out["grid_barrier_us_128_ctas"] = (time.perf_counter() - t0) * 1e6 / 20000
    best = "graph" if out["us_per_step_graph"] <= out["us_per_step_cooperative"] else "cooperative"
    lat = P.Lattice([P.Member(n, n, tau)], precision=64, diag_every=D,
                    graph_steps=16 if best == "graph" else 0, stream=stream, device=dev)
    lat.init_fields(0, rho, ux, uy)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps // D):
        lat.step(D)
        st = lat.subvolume_balance(0, Ls)
    torch.cuda.synchronize()
    out["workload_ms"] = (time.perf_counter() - t0) * 1e3
    out["workload_stepping"] = best
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

    cpl = {}

    def timed(q):
        lat = P.Lattice3D([P.Member3(n, n, n, 0.52)] * M, precision=32, stream=stream, device=dev,
                          lattice=q)
        cpl[q] = lat.tuning()["cells_per_lane"]
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
            "cells_per_lane": cpl[19],
            "d3q27": {"glups": glups27, "bytes_per_lu": 216, "achieved_gbs": gbs27,
                      "frac": gbs27 / peak, "cells_per_lane": cpl[27]},
            "diagnostic_event_ms_fp64_64cubed_all_origins": 1e3 * diag_s,
            "diagnostic_event_ms_fp32_64cubed_all_origins": 1e3 * diag32_s}


def alu_peaks(P, stream):
    """Measured FMA throughput of this GPU (TFLOP/s, two flops per FMA):
    the ceiling of the kernels bounded by arithmetic rather than HBM."""
    return {"fp64_tflops": P.probe_fma_rate(64, stream) / 1e12,
            "fp32_tflops": P.probe_fma_rate(32, stream) / 1e12,
            "how": "lbm_probe_fma_rate: 8 independent FMA chains per thread, 8 x 256-thread "
                   "CTAs per SM, CUDA events"}


def fp64_instruction_counts():
    """FP64 flops and FP64 instructions per lattice update of the FP64
    kernels (dadd + dmul + 2 dfma, and dadd + dmul + dfma, ncu counters)
    from the committed summary, valid only while the kernel sources are
    unchanged."""
    p = os.path.join(ROOT, "profiles", "fp64_flops_per_lu.json")
    if not os.path.exists(p):
        return {}
    with open(p) as fh:
        d = json.load(fh)
    out = {}
    for name, rec in d.get("kernels", {}).items():
        src = os.path.join(ROOT, "paper_1809_06735_gb300", "csrc", rec["source"])
        with open(src, "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] == rec.get("source_sha256_16"):
                out[name] = (rec["fp64_flops_per_lu"], rec["fp64_instr_per_lu"])
    return out


def issue_counts():
    """Warp instructions per lattice update of the issue-bound kernels
    (sm__inst_executed.sum over the launch's cells, ncu) from the committed
    summary, valid only while the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "elbm_issue.json")
    if not os.path.exists(p):
        return {}
    with open(p) as fh:
        d = json.load(fh)
    out = {}
    for name, rec in d.get("kernels", {}).items():
        src = os.path.join(ROOT, "paper_1809_06735_gb300", "csrc", rec["source"])
        with open(src, "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] == rec.get("source_sha256_16"):
                out[name] = rec["warp_instr_per_lu"]
    return out


def issue_peak(dev_index=0):
    """Peak instruction issue of the GPU: 4 schedulers per SM, one warp
    instruction each per clock, at the maximum SM clock (warp instr/s)."""
    import torch
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    return 4.0 * sms * mhz * 1e6


def fp64_roofline(counts, glups, peaks):
    """The FP64-pipe roofline of a kernel from its counted flops and
    instructions per update: achieved flop rate against the measured FMA
    rate, and the pipe's instruction rate against the FMA chains' (an add or
    a multiply occupies the pipe like an FMA)."""
    flops, instr = counts
    tf = flops * glups / 1e3
    return {"bound": "fp64", "fp64_flops_per_lu": flops, "fp64_instr_per_lu": instr,
            "achieved": tf, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
            "frac": tf / peaks["fp64_tflops"],
            "pipe_instr_frac": instr * glups * 1e9 / (peaks["fp64_tflops"] * 1e12 / 2)}


def fp64_plain_leg(P, stream, dev, peak_hbm, peaks, dev_fields=None):
    """The plain single-instance FP64 step (double buffer, general kernel)
    on one 4096^2 member (2 x 1.2 GB of populations: far beyond the L2, so
    the HBM figure means something), against both bounds: 144 algorithmic
    bytes per update over the measured copy bandwidth, and the FP64 flops
    per update (ncu counters) over the measured FP64 FMA rate."""
    import torch
    n = 4096
    lat = P.Lattice([P.Member(n, n, 0.52)], precision=64, graph_steps=10, stream=stream,
                    device=dev)
    u = li.smooth_fields(n, n, seed=11, amp=0.02, kmax=16)
    v = li.smooth_fields(n, n, seed=12, amp=0.02, kmax=16)
    lat.init_fields(0, np.ones((n, n)), u, v)
    lat.step(10)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    lat.step(20)
    b.record(stream)
    torch.cuda.synchronize()
    secs = a.elapsed_time(b) / 1e3 / 20
    lat.close()
    glups = n * n / secs / 1e9
    gbs = BYTES_PER_LU_F64 * glups
    counts = fp64_instruction_counts().get("k_step_scalar<double>")
    out = {"grid": [n, n], "glups": glups, "bytes_per_lu": BYTES_PER_LU_F64,
           "achieved_gbs": gbs, "hbm_frac": gbs / peak_hbm}
    if counts is not None:
        out["fp64_roofline"] = fp64_roofline(counts, glups, peaks)
    return out


def forced_sweep_leg(P, stream, dev, peak):
    """The forced tau-sweep: 15 FP32 members {256, 512, 1024}^2 x tau
    {0.505, 0.51, 0.52, 0.55, 0.6}, Kolmogorov kf = 4 with drag 1e-4, all in
    one launch per step (uneven tile table).  One diagnostic period of 200
    steps: the stream-collide rate (aggregate, and per member: each member
    advances the same 200 steps in the batch's time) and its roofline, then
    the balance event of every member at L = 2..512 (L > N skipped) over
    every periodic origin, timed on its own."""
    import torch
    wl = li.forced_sweep_workload()
    mem = wl["members"]
    lat = P.Lattice([P.Member(m["n"], m["n"], m["tau"], 1.0, 1, m["kf"], m["F0"], m["alpha"])
                     for m in mem], precision=32, diag_every=PERIOD, graph_steps=PURE_STEPS - 1,
                    stream=stream, device=dev)
    for i, m in enumerate(mem):
        lat.init_fields(i, *li.random_phase(m["n"], seed=m["seed"], u_rms=wl["u_rms"]))
    cells = [m["n"] * m["n"] for m in mem]
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    lat.step(PERIOD)  # warm-up period (graphs, snapshots)
    lat.subvolume_balance_batch(range(len(mem)), wl["Ls"])
    a, b, c, d = ev(), ev(), ev(), ev()
    torch.cuda.synchronize()
    a.record(stream)
    lat.step(PURE_STEPS)
    b.record(stream)
    lat.step(PERIOD - PURE_STEPS)
    c.record(stream)
    st = lat.subvolume_balance_batch(range(len(mem)), wl["Ls"])
    d.record(stream)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(st[:, 0, 2:, 0]))
    pure_s = a.elapsed_time(b) / 1e3 / PURE_STEPS
    period_s = a.elapsed_time(c) / 1e3
    event_s = c.elapsed_time(d) / 1e3
    tot = sum(cells)
    glups = tot / pure_s / 1e9
    gbs = BYTES_PER_LU_F32 * glups
    lat.close()
    return {"members": len(mem), "cells": tot, "glups": glups,
            "per_member_glups": [{"n": m["n"], "tau": m["tau"], "glups": c_ / pure_s / 1e9}
                                 for m, c_ in zip(mem, cells)],
            "bytes_per_lu": BYTES_PER_LU_F32, "achieved_gbs": gbs, "frac": gbs / peak,
            "diagnostic_event_ms_all_origins": 1e3 * event_s, "sizes": list(wl["Ls"]),
            "glups_with_diagnostic": tot * PERIOD / (period_s + event_s) / 1e9}


def large_grid_leg(P, stream, dev, peak):
    """The large single forced run: one FP32 member of 8192^2, tau 0.51,
    Kolmogorov kf = 4, drag 1e-5 (smooth seeded initial fields), its
    stream-collide rate and roofline, and one balance event at
    L = 2..4096 over all 67 M periodic origins (FP64 statistics), timed on
    its own and folded into a 100-step diagnostic period."""
    import torch
    wl = li.large_forced_workload()
    n, D = wl["n"], wl["diag_every"]
    lat = P.Lattice([P.Member(n, n, wl["tau"], 1.0, 1, wl["kf"], wl["F0"], wl["alpha"])],
                    precision=32, diag_every=D, graph_steps=D - 4, stream=stream, device=dev)
    r = 1.0 + li.smooth_fields(n, n, seed=7, amp=1e-3, kmax=16)
    u = li.smooth_fields(n, n, seed=5, amp=0.03, kmax=16)
    v = li.smooth_fields(n, n, seed=6, amp=0.03, kmax=16)
    lat.init_fields(0, r, u, v)
    del r, u, v
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    lat.step(D)
    lat.subvolume_balance(0, wl["Ls"])  # warm-up event
    a, b, c, d = ev(), ev(), ev(), ev()
    torch.cuda.synchronize()
    a.record(stream)
    lat.step(D - 3)
    b.record(stream)
    lat.step(3)
    c.record(stream)
    st = lat.subvolume_balance(0, wl["Ls"])
    d.record(stream)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(st[:, 2:, 0]))
    pure_s = a.elapsed_time(b) / 1e3 / (D - 3)
    glups = n * n / pure_s / 1e9
    gbs = BYTES_PER_LU_F32 * glups
    event_s = c.elapsed_time(d) / 1e3
    period_s = a.elapsed_time(c) / 1e3
    lat.close()
    return {"grid": [n, n], "glups": glups, "bytes_per_lu": BYTES_PER_LU_F32,
            "achieved_gbs": gbs, "frac": gbs / peak, "sizes": list(wl["Ls"]),
            "diagnostic_event_ms_all_origins": 1e3 * event_s,
            "boxes_per_event": n * n * len(wl["Ls"]),
            "glups_with_diagnostic": n * n * D / (period_s + event_s) / 1e9}


def adjoint_leg(P, stream, dev, peaks):
    """The differentiation workload: 256^2, tau 0.55, Kolmogorov kf = 4
    (drag 1e-4), J = mean over n in [1000, 2000] of the L = 16 box average
    of the dissipation term, checkpoints every 100 steps; the forward pass
    (with checkpoints and the objective) and the reverse pass (recomputation
    of each interval + adjoint sweep) timed end to end with FP64 and FP32
    forward states, and the adjoint step kernel alone (216 algorithmic bytes
    per update: the state, the adjoint pulled from the neighbours, the new
    adjoint; FP64 arithmetic)."""
    import torch
    from paper_1809_06735_gb300.adjoint import ObjectiveSpec, adjoint_objective, forward_objective
    wl = li.adjoint_workload()
    n, tau, F0 = wl["n"], wl["tau"], wl["F0"]
    init = P.Lattice([P.Member(n, n, tau)], precision=64, stream=stream, device=dev)
    init.init_fields(0, *li.random_phase(n, seed=wl["seed"], u_rms=wl["u_rms"]))
    f0 = init.get_populations(0).clone()
    init.close()
    out = {"grid": [n, n], "window": [wl["n0"], wl["n1"]], "L": wl["L"],
           "checkpoint_every": wl["checkpoint_every"]}
    for prec in (64, 32):
        # untimed warm-up on a short window: the first forward of a process
        # pays one-off set-up (about 0.25 s on the first FP64 one)
        short = ObjectiveSpec(nx=n, ny=n, kf=wl["kf"], alpha=wl["alpha"], n0=10, n1=20,
                              box=wl["box"], L=wl["L"], precision=prec, checkpoint_every=10)
        _, warm_ckpts, warm = forward_objective(short, tau, F0, f0, keep_checkpoints=True)
        adjoint_objective(short, tau, F0, warm, warm_ckpts)
        warm.close()
        spec = ObjectiveSpec(nx=n, ny=n, kf=wl["kf"], alpha=wl["alpha"], n0=wl["n0"],
                             n1=wl["n1"], box=wl["box"], L=wl["L"], precision=prec,
                             checkpoint_every=wl["checkpoint_every"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, ckpts, lat = forward_objective(spec, tau, F0, f0, keep_checkpoints=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        dtau, dF0, _ = adjoint_objective(spec, tau, F0, lat, ckpts)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        lat.close()
        out["fp%d_forward" % prec] = {
            "J": float(J), "dJ_dtau": float(dtau), "dJ_dF0": float(dF0),
            "forward_ms": 1e3 * (t1 - t0), "forward_us_per_step": 1e6 * (t1 - t0) / wl["n1"],
            "reverse_ms": 1e3 * (t2 - t1),
            "reverse_us_per_step": 1e6 * (t2 - t1) / (wl["n1"] + 1)}
    # the adjoint step kernel alone: a sweep over 100 recorded states
    lat = P.Lattice([P.Member(n, n, tau, 1.0, 1, wl["kf"], F0, wl["alpha"])], precision=64,
                    stream=stream, device=dev)
    lat.set_populations(0, f0)
    K = 100
    states = torch.empty((K, 9, n, n), dtype=torch.float64, device=dev)
    lat.record_trajectory(0, states)
    lam_in = torch.randn((9, n, n), dtype=torch.float64, device=dev) * 1e-3
    lam_out, lam_tmp = torch.empty_like(lam_in), torch.empty_like(lam_in)
    acc = torch.zeros(2, dtype=torch.float64, device=dev)
    zero = np.zeros(K)
    lat.adjoint_sweep(0, states, lam_in, lam_out, lam_tmp, zero, (0, 0), 1, acc[0:1], acc[1:2])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    lat.adjoint_sweep(0, states, lam_in, lam_out, lam_tmp, zero, (0, 0), 1, acc[0:1], acc[1:2])
    b.record(stream)
    torch.cuda.synchronize()
    lat.close()
    step_s = a.elapsed_time(b) / 1e3 / K
    glups = n * n / step_s / 1e9
    k = {"us_per_step": 1e6 * step_s, "glups": glups, "bytes_per_lu": 216,
         "achieved_gbs": 216 * glups,
         "note": "256^2 FP64: 14 MB per step, L2-resident; one k_adjoint launch per step, "
                 "the gradient reduction (k_adjoint_final) once per 100-step sweep"}
    counts = fp64_instruction_counts().get("k_adjoint")
    if counts is not None:
        k["fp64_roofline"] = fp64_roofline(counts, glups, peaks)
    out["adjoint_kernel"] = k
    return out


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
# shapes x 8 launches, then the 3 fastest again 3 x 14 launches each, so 414
# launches of k_step_f32_vec come before the first step of the run.
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
    autotuner's 414 launches and the 64 initialisations come first."""
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


def case_diag_large(P, n=8192, events=2):
    """The large forced run's balance event: one FP32 member of 8192^2,
    L = 2..4096 over every periodic origin (805 M boxes), twice (about
    31 GB of device memory)."""
    import torch
    wl = li.large_forced_workload()
    lat = P.Lattice([P.Member(n, n, wl["tau"], 1.0, 1, wl["kf"], wl["F0"], wl["alpha"])],
                    precision=32, diag_every=4)
    lat.init_fields(0, 1.0 + li.smooth_fields(n, n, seed=7, amp=1e-3, kmax=16),
                    li.smooth_fields(n, n, seed=5, amp=0.03, kmax=16),
                    li.smooth_fields(n, n, seed=6, amp=0.03, kmax=16))
    for _ in range(events):
        lat.step(4)
        stats = lat.subvolume_balance(0, wl["Ls"])
    torch.cuda.synchronize()
    assert np.all(np.isfinite(stats[:, 2:, 0]))
    print("diag_large case done:", lat.launch_count, "launches")


def case_diag_query(P, n=2048, events=2):
    """The all-origins box query on tables larger than L2: one FP32 member of
    2048^2 (12 corner tables of 4.2 M records, 400 MB), L = 2..2048 over
    every periodic origin (46 M boxes per event)."""
    import torch
    wl = li.large_forced_workload()
    lat = P.Lattice([P.Member(n, n, wl["tau"], 1.0, 1, wl["kf"] * n // wl["n"], wl["F0"],
                              wl["alpha"])], precision=32, diag_every=4)
    lat.init_fields(0, 1.0 + li.smooth_fields(n, n, seed=7, amp=1e-3, kmax=32),
                    li.smooth_fields(n, n, seed=5, amp=0.03, kmax=32),
                    li.smooth_fields(n, n, seed=6, amp=0.03, kmax=32))
    Ls = [L for L in wl["Ls"] if L <= n]
    for _ in range(events):
        lat.step(4)
        stats = lat.subvolume_balance(0, Ls)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(stats[:, 2:, 0]))
    print("diag_query case done:", lat.launch_count, "launches")


def case_fp64(P, n=512, steps=20):
    import torch
    lat = P.Lattice([P.Member(n, n, 0.52)], precision=64)
    lat.init_fields(0, *li.random_phase(n, seed=1000, u_rms=0.02))
    lat.step(steps)
    torch.cuda.synchronize()
    print("fp64 case done")


def case_taylor_green(P, events=3):
    """The FP64 Taylor-Green workload (64^2, tau 0.6) for a few of its
    balance events: 100 steps, then the balance at L in {4, 8, 16, 32} over
    every origin, per event."""
    import torch
    wl = li.taylor_green_workload()
    n, tau, D, Ls = wl["n"], wl["tau"], wl["diag_every"], wl["Ls"]
    lat = P.Lattice([P.Member(n, n, tau)], precision=64, diag_every=D, graph_steps=16)
    lat.init_fields(0, *li.taylor_green(n, u0=wl["u0"]))
    for _ in range(events):
        lat.step(D)
        lat.subvolume_balance(0, Ls)
    torch.cuda.synchronize()
    print("taylor green case done:", lat.launch_count, "launches")


def case_adjoint(P, n=256, steps=6):
    import torch
    F0 = li.kolmogorov_F0(n, 0.55, 4, 1e-4, 0.03)
    lat = P.Lattice([P.Member(n, n, 0.55, 1.0, 1, 4, F0, 1e-4)], precision=64)
    lat.init_fields(0, *li.random_phase(n, seed=0, u_rms=0.02))
    acc = torch.zeros(2, dtype=torch.float64, device="cuda")
    lat.objective_steps(0, steps, 1e-3, (0, 0), 16, acc[0:1])  # forward objective levels
    f = lat.get_populations(0)
    lam = torch.zeros_like(f)
    out = torch.empty_like(f)
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
    peaks_alu = alu_peaks(P, stream)
    fp64_big = fp64_plain_leg(P, stream, dev, peak, peaks_alu)
    forced_sweep = forced_sweep_leg(P, stream, dev, peak)
    large_grid = large_grid_leg(P, stream, dev, peak)
    adjoint = adjoint_leg(P, stream, dev, peaks_alu)
    paper_forcing = paper_forcing_leg(P, stream, dev, measured_peaks()[0])
    tau_trend = forced_tau_trend_leg(P, stream, dev)
    collisions = collision_models_leg(P, stream, dev, measured_peaks()[0])
    three_d = three_d_leg(P, stream, dev, measured_peaks()[0])
    taylor_green = taylor_green_leg(P, stream, dev)

    # end to end through the public API with host buffers: every step passes
    # the pinned host initial fields of all members to lbm_init_fields_batch
    # (the initialisation kernel reads them in place over the host link, no
    # staging copy), runs the period and reads its statistics back to pinned
    # host memory.  Pipelined as a production caller would: step k-1's
    # statistics travel to the host (copy stream) while step k steps; the
    # diagnostic runs on the library's diagnostic stream.
    e2e_steps = max(1, args.steps)
    copy_stream = torch.cuda.Stream(device=dev)
    host_stats = torch.empty((e2e_steps + 1, M, len(Ls), 15, 2), dtype=torch.float64,
                             pin_memory=True)
    e2e_buf = [torch.empty((M, len(Ls), 15, 2), dtype=torch.float64, device=dev)
               for _ in range(2)]

    def e2e_run(nsteps, record):
        for k in range(nsteps):
            lat.init_fields_batch(all_members, host[0], host[1], host[2])
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
    runs = []
    gc.collect()
    gc.disable()  # as in the timed steps above
    for _ in range(3):  # median of three pipelined runs: host-side jitter is one-sided
        torch.cuda.synchronize()
        te = time.perf_counter()
        e2e_run(e2e_steps, host_stats)
        torch.cuda.synchronize()
        runs.append(time.perf_counter() - te)
    gc.enable()
    assert np.all(np.isfinite(host_stats[:e2e_steps, :, :, 2:, 0].numpy()))
    te = float(np.median(runs))
    if ws > 1:
        te = max_over_ranks(te)
    e2e = {"value": ws * lu_per_gpu_step * e2e_steps / te / 1e9, "unit": "GLUPS",
           "h2d_bytes_per_step": int(M * 3 * n * n * 8),
           "d2h_bytes_per_step": int(M * len(Ls) * 30 * 8),
           "note": "per step: the pinned host fields of all members passed as host pointers "
                   "to lbm_init_fields_batch (read in place by the initialisation kernel), "
                   "200 steps, Table 1 statistics to pinned host memory; step k-1's "
                   "statistics travel while step k runs; wall clock over %d steps including "
                   "pipeline fill and drain, median of 3 runs (%s ms)"
                   % (e2e_steps, ", ".join("%.1f" % (1e3 * r) for r in runs))}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_all_cores()

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
                                           "ratio_batched_fp32_over_fp64": step_glups / fp64_glups,
                                           "roofline_4096sq": fp64_big},
            "alu_peaks": peaks_alu,
            "forced_sweep_15_uneven": forced_sweep,
            "large_forced_8192sq": large_grid,
            "adjoint_256sq": adjoint,
            "paper_forcing_ensemble": paper_forcing,
            "forced_tau_sweep_trend": tau_trend,
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
