#!/usr/bin/env python
"""Benchmark of the block-forest DG hot path (compressible Euler, SSP-RK3).

Workload (default): 3D Euler on a jittered unit cube of 8 rotated hex root
blocks with 8^3-cell blocks and two static refinement levels (71 leaves,
36,352 cells), p = 2 (27 modes x 5 variables), isentropic vortex scaled into
the cube, CFL 0.1; the FP32 form is the reported line, the FP64 form is
measured beside it.  One step = one SSP-RK3 time increment (3 stages of
guard fill + fused residual / inverse mass / stage combination, CFL minimum
on the last stage).  Metric: DG DOF-updates per second per RK stage
(= DOF x 3 x steps / time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                 [--workload jitter3d|jitter3dp1|jitter3dp3|cube8|cube8p1|cube8p3]
                 [--nonconforming paper|mortar]
  python bench.py --serve [--serve-requests R] [--serve-active A]
  python bench.py --amr [--steps K]          (K regrid periods of 10 steps)

Timing: CUDA events on the forest's stream around each step, an L2 flush
(256 MiB write) before every timed step, warm-up steps first, barrier and
max over ranks.  Multi-GPU: independent replicas (the path has no exchange
step on one GPU); value = sum over ranks.  --impl reference times the FP64
CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOAD = "3d-euler-jittered-cube-8roots-71leaves-n8-p2"
HBM_FALLBACK = 6800.0
# DRAM bytes (read + write) per stage-kernel launch, averaged over the three
# stages of one time step (ncu dram__bytes_read.sum + dram__bytes_write.sum,
# cold L2), by (workload, stage kernel), for the kernels as they are now; a
# workload without a capture of the current kernel reports null.  The 16^3
# cube at p = 2 is 8 x the 512-leaf cube's figure (same kernel, tiling and
# grid of one CTA per work item, state above L2 in both, traffic
# proportional to the leaves: 377.0 MB there, the algorithmic 377.5 MB); the
# 512-leaf cube at p = 1 fits L2, so no figure is scaled to the 16^3 cube at
# p = 1.
STAGE_TRAFFIC_BYTES = {("jitter3d", "pair"): 47.8e6, ("cube16p2", "pair"): 8 * 377.0e6}
TRAFFIC_HOW = "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, cold L2, mean of the 3 stages of a step"


def stage_kernel_name(f, p):
    """The stage kernel the forest's time step launches (after tuning)."""
    k = f.tuning()["stage_kernel"]
    if k == "pair":
        return f"k_stage_pair<{p}>"
    if k == "pair5":
        return f"k_stage_pair<{p}> (five CTAs per SM)"
    return f"k_stage<3,{p},8,float>"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": HBM_FALLBACK}, "fallback"


WORKLOADS = {
    # the benchmark line: 71 leaves, 36,352 cells, p=2
    "jitter3d": (WORKLOAD, lambda: W.jitter3d_forest(seed=0), 2),
    # larger affine case for profiling (state 141 MB FP32, above L2)
    "cube8": ("3d-euler-periodic-cube-8^3-roots-n8-p2", lambda: W.periodic_cube_forest(8), 2),
    "cube8p1": ("3d-euler-periodic-cube-8^3-roots-n8-p1", lambda: W.periodic_cube_forest(8), 1),
    "cube8p3": ("3d-euler-periodic-cube-8^3-roots-n8-p3", lambda: W.periodic_cube_forest(8), 3),
    "cube16p1": ("3d-euler-periodic-cube-16^3-roots-n8-p1", lambda: W.periodic_cube_forest(16), 1),
    "cube16p2": ("3d-euler-periodic-cube-16^3-roots-n8-p2", lambda: W.periodic_cube_forest(16), 2),
    "jitter3dp1": ("3d-euler-jittered-cube-8roots-71leaves-n8-p1", lambda: W.jitter3d_forest(seed=0), 1),
    "jitter3dp3": ("3d-euler-jittered-cube-8roots-71leaves-n8-p3", lambda: W.jitter3d_forest(seed=0), 3),
}
_SEL = ["jitter3d"]
_NC = ["paper"]  # level-jump treatment: the paper's guard scheme or the mortar repair


def the_workload():
    name, mk, p = WORKLOADS[_SEL[0]]
    return mk(), p


def vortex(x):
    return W.isentropic_vortex(x, scale=10.0)


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------- dist
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def barrier_max(x, ws):
    """Max of x over the ranks (the slowest replica sets the job time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ms_local, ws):
    """Whole-job rate of ws independent replicas: all ranks' units over the
    max-over-ranks time (replicas do identical work, so units scale by ws)."""
    ms = barrier_max(ms_local, ws)
    return units_per_rank * ws / (ms / 1e3), ms


# ---------------------------------------------------------------- CPU legs
def _oracle_worker(rank, nworkers, nleaves, reps, barrier, queue):
    """One process of the oracle timing: builds the FP64 oracle on the bench
    workload, then (after every process has built it) times `reps` SSP-RK3
    stages (guard fill + residual + mass solve + update) on its share of the
    first `nleaves` leaves.  Runs in a spawned process."""
    from oracle import dg, forest as FO
    S = dg.Solver(FO.build(W.jitter3d_forest(seed=0)), 2, cfl=0.1)
    U = S.project(vortex)
    mine = list(range(rank, nleaves, nworkers))
    spans = []
    for _ in range(reps):
        barrier.wait()
        t0 = time.time()
        if mine:
            L = S.residual(U, leaves=mine)
            V = U[mine] + 1e-4 * L[mine]  # noqa: F841  (the stage update of those leaves)
        spans.append((t0, time.time()))
    dof = len(mine) * S.nv * S.ops.M * S.n ** S.d
    queue.put((rank, spans, dof))


def oracle_timing(nworkers, nleaves, reps):
    """Time the oracle with `nworkers` spawned processes (one thread each,
    leaves dealt round robin).  Returns per-repetition wall times (max end -
    min start over the processes) and the DOF updated per repetition."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(nworkers), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(r, nworkers, nleaves, reps, barrier, queue))
             for r in range(nworkers)]
    for pr in procs:
        pr.start()
    res = [queue.get(timeout=1800) for _ in procs]
    for pr in procs:
        pr.join()
    walls = [max(r[1][i][1] for r in res) - min(r[1][i][0] for r in res) for i in range(reps)]
    return walls, sum(r[2] for r in res)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline():
    """The oracle as it stands on the host cores: one thread, and one process
    per core parallel over leaves (the core count is stated)."""
    cores = host_cores()
    w1, dof = oracle_timing(1, 71, 1)
    wa, dofa = oracle_timing(cores, 71, 2)
    v1 = dof / w1[0]
    va = dofa * len(wa) / sum(wa)
    return {"value": va, "unit": "DOF-updates/s", "cores": cores, "nproc": os.cpu_count(), "kind": "oracle",
            "value_1_thread": v1,
            "sample": (f"one SSP-RK3 stage (guard fill + residual + mass solve + update) of the full 71-leaf "
                       f"workload in FP64: {w1[0]:.1f} s on 1 thread; {len(wa)} stages on {cores} processes "
                       f"(one thread each, leaves dealt round robin), {sum(wa):.1f} s")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    # each step: one SSP-RK3 stage on all host cores; the leaf sample is the
    # whole workload unless that would take more than a few minutes
    cores = host_cores()
    per_leaf = 0.25 / cores
    budget = 150.0
    nleaves = int(max(cores, min(71, budget / max(1, args.steps + args.warmup) / per_leaf)))
    nleaves = min(nleaves, 71)
    walls, dof = oracle_timing(cores, nleaves, args.steps + args.warmup)
    times = walls[args.warmup:]
    t = sum(times)
    value = dof * len(times) / t
    line = {"impl": "reference", "metric": "DG DOF-updates/s per RK stage", "value": value,
            "unit": "DOF-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_leaves": nleaves},
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": cores, "nproc": os.cpu_count(),
                             "kind": "oracle",
                             "sample": (f"one SSP-RK3 stage per step on {nleaves} of the 71 leaves, FP64, "
                                        f"{cores} processes of one thread, leaves dealt round robin")},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU leg
def timed_steps(f, steps, stream, flush, torch):
    """Sum of per-step event times on the forest's stream, L2 flushed between."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            f.rk_step()
            evs[i][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def run_ours(args):
    import torch
    import paper_2502_12620_gb300 as pkg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    pk, pk_kind = peaks()
    w, p = the_workload()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def make(prec):
        f = pkg.Forest.from_workload(w, p=p, precision=prec, device=local, cfl=0.1, nonconforming=_NC[0])
        f.set_stream(stream)
        f.project(vortex)
        return f

    f32 = make({"fp32": pkg.FP32, "fp64": pkg.FP64, "fp32_comp": pkg.FP32_COMP}[args.precision] if args.quick
               else pkg.FP32)
    dof = f32.n_leaves * f32.nv * f32.M * f32.nc
    U0 = f32.get_state()
    for _ in range(args.warmup):
        f32.rk_step()
    if ws > 1:
        torch.distributed.barrier()
    with Clocks(local) as ck:
        ms = timed_steps(f32, args.steps, stream, flush, torch)
    value, ms = job_throughput(dof * 3 * args.steps, ms, ws)
    status = f32.status_word()
    if args.quick:
        if rank == 0:
            print(json.dumps({"workload": WORKLOADS[_SEL[0]][0], "precision": args.precision, "value": value,
                              "unit": "DOF-updates/s", "tuning": f32.tuning(),
                              "ms_per_step": ms / args.steps, "dof": dof, "status_word": status,
                              "nonconforming": _NC[0], "clocks": ck.summary()}))
        return 0

    # instrumented replay of the same steps: per-kernel durations
    f32.set_state(U0)
    f32.set_time(0.0)
    f32.set_timing(True)
    for _ in range(args.warmup):
        f32.rk_step()
    f32.kernel_times()
    timed_steps(f32, args.steps, stream, flush, torch)
    kt = f32.kernel_times()
    f32.set_timing(False)
    stage_ms, stage_n = kt["stage"]
    nL, nc, NG = f32.n_leaves, f32.nc, 21
    state_bytes_avg = dof * 4 * (2 + 3 + 3) / 3.0
    geo_bytes = nL * nc * NG * 4 + nL * nc * 4 / 3.0
    alg_bytes = state_bytes_avg + geo_bytes
    achieved = alg_bytes / (stage_ms / stage_n / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"],
            "traffic": STAGE_TRAFFIC_BYTES.get((_SEL[0], f32.tuning()["stage_kernel"])),
            "traffic_how": TRAFFIC_HOW,
            "kernel": stage_kernel_name(f32, p),
            "bytes_per_launch": alg_bytes, "avg_launch_us": 1e3 * stage_ms / stage_n,
            "peak_source": pk_kind,
            "other_kernels_us_per_step": {"guard": 1e3 * kt["guard"][0] / args.steps,
                                          "dt": 1e3 * kt["dt"][0] / args.steps}}

    # FP64 form of the same workload
    f64 = make(pkg.FP64)
    for _ in range(max(1, args.warmup // 2)):
        f64.rk_step()
    k64 = max(2, min(args.steps, 10))
    ms64 = barrier_max(timed_steps(f64, k64, stream, flush, torch), ws)
    value64 = dof * 3 * k64 / (ms64 / 1e3) * ws

    # compensated FP32 (FP64 state, FP32 residual and increments)
    fc = make(pkg.FP32_COMP)
    for _ in range(max(1, args.warmup // 2)):
        fc.rk_step()
    kc = max(2, min(args.steps, 10))
    msc = barrier_max(timed_steps(fc, kc, stream, flush, torch), ws)
    valuec = dof * 3 * kc / (msc / 1e3) * ws

    # accuracy: FP32 and compensated FP32 vs FP64 after the same steps from the same state
    f32.set_timing(False)
    a32 = make(pkg.FP32)
    a64 = make(pkg.FP64)
    ac = make(pkg.FP32_COMP)
    nacc = 20
    for _ in range(nacc):
        a32.rk_step()
        a64.rk_step()
        ac.rk_step()
    s32 = a32.get_state().astype(np.float64)
    s64 = a64.get_state()
    sc = ac.get_state()
    l2 = float(np.linalg.norm(s32 - s64) / np.linalg.norm(s64))
    linf = float(np.max(np.abs(s32 - s64)) / np.max(np.abs(s64)))
    l2c = float(np.linalg.norm(sc - s64) / np.linalg.norm(s64))
    linfc = float(np.max(np.abs(sc - s64)) / np.max(np.abs(s64)))

    # end to end through the public API with host buffers (pinned)
    host = torch.empty(U0.size, dtype=torch.float32).pin_memory().numpy().reshape(U0.shape)
    host[...] = U0
    e = make(pkg.FP32)
    for _ in range(2):
        e.set_state(host)
        e.rk_step()
        e.get_state(host)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e.set_state(host)
        e.rk_step()
        e.get_state(host)
    torch.cuda.synchronize()
    te = barrier_max(time.perf_counter() - t0, ws)
    e2e = {"value": dof * 3 * args.steps / te * ws, "unit": "DOF-updates/s",
           "h2d_bytes_per_step": int(U0.nbytes), "d2h_bytes_per_step": int(U0.nbytes)}

    if rank != 0:
        return 0
    line = {
        "metric": "DG DOF-updates/s per RK stage", "value": value, "unit": "DOF-updates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[_SEL[0]][0], "leaves": nL, "cells": nL * nc, "p": p, "dof": dof,
                   "precision": "fp32", "l2_flush": "256 MiB write before every timed step",
                   "nonconforming": _NC[0], "parallelism": f"replicas x{ws}"},
        "roofline": roof,
        "fp64": {"value": value64, "unit": "DOF-updates/s", "ms_per_step": ms64 / k64, "steps": k64},
        "fp32_comp": {"value": valuec, "unit": "DOF-updates/s", "ms_per_step": msc / kc, "steps": kc},
        "accuracy": {"steps": nacc, "l2_rel_fp32_vs_fp64": l2, "linf_rel_fp32_vs_fp64": linf,
                     "l2_rel_fp32_comp_vs_fp64": l2c, "linf_rel_fp32_comp_vs_fp64": linfc},
        "e2e": e2e,
        "clocks": ck.summary(),
        "gpu_launches": int(sum(c for _, c in kt.values())),
        "tuning": f32.tuning(),
        "status_word": status,
    }
    if not args.quick_line:
        # affine periodic cubes far above L2 (each state copy 0.34 / 1.13 GB)
        line["over_l2"] = {k: over_l2_case(k, args, stream, flush, pk, pk_kind, torch, pkg) for k in OVER_L2}
        line["batch"] = {}
        for q in (1, 2):
            try:
                line["batch"][f"p{q}"] = batch_case(q, args, flush, pk, pk_kind, torch, pkg)
            except pkg.DgfError as e:  # reported, not hidden
                line["batch"][f"p{q}"] = {"error": str(e)}
        line["serve"] = run_serve(args, sub=True)
        line["amr"] = {}
        for q in (1, 3):
            try:
                line["amr"][f"p{q}"] = run_amr(args, sub=True, p=q,
                                                periods=args.amr_sub_periods if q < 3 else args.amr_sub_periods // 2)
            except pkg.DgfError as e:  # a run that breaks down is reported, not hidden
                line["amr"][f"p{q}"] = {"error": str(e)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line))
    return 0


# the batched path: one batch of three affine periodic cubes of 8^3, 10^3 and
# 12^3 roots (3,240 blocks; 0.27 GB per state copy at p = 1, 0.9 GB at p = 2)
BATCH_CUBES = (8, 10, 12)


def batch_case(p, args, flush, pk, pk_kind, torch, pkg):
    """DOF-updates/s of one batch of the BATCH_CUBES forests advanced together
    (one launch per kernel and stage for all three, one CUDA graph per time
    increment, L2 flushed between timed steps, CUDA events on the batch
    stream) and the step's fraction of the measured copy peak: the three
    stage launches' algorithmic bytes (as for a single forest) over the whole
    step, guard traces and time increments included, so a lower bound of the
    batch stage kernel's own fraction."""
    stream = torch.cuda.Stream()
    fs = []
    for B in BATCH_CUBES:
        f = pkg.Forest.from_workload(W.periodic_cube_forest(B), p=p, precision=pkg.FP32, cfl=0.1)
        f.set_state_nodal(vortex(f.quad_points()))
        fs.append(f)
    b = pkg.Batch(stream=stream)
    b.set(fs, [1e9] * len(fs))
    b.step(args.warmup)
    b.sync()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            b.step(1)
            evs[i][1].record(stream)
    stream.synchronize()
    ms = sum(a.elapsed_time(c) for a, c in evs)
    dof = sum(f.n_leaves * f.nv * f.M * f.nc for f in fs)
    cells = sum(f.n_leaves * f.nc for f in fs)
    alg_step = dof * 4 * (2 + 3 + 3) + cells * 4
    achieved = alg_step / (ms / args.steps / 1e3) / 1e9
    out = {"workload": f"batch-of-3-periodic-cubes-{'-'.join(f'{B}^3' for B in BATCH_CUBES)}-roots-n8-p{p}",
           "members": len(fs), "blocks": sum(f.n_leaves for f in fs), "p": p, "dof": dof,
           "value": dof * 3 * args.steps / (ms / 1e3), "unit": "DOF-updates/s", "ms_per_step": ms / args.steps,
           "steps": args.steps,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved / pk["hbm_gbs"], "traffic": None, "peak_source": pk_kind,
                        "scope": "whole batch step (3 stage launches, 3 guard launches, the dt launch)",
                        "bytes_per_step": alg_step},
           "status_words": [f.status_word() for f in fs]}
    b.close()
    for f in fs:
        f.close()
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    """The bench line's batched-path records alone (rank 0 at N = 1 prints
    one JSON line per degree)."""
    import torch
    import paper_2502_12620_gb300 as pkg
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pk, pk_kind = peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for q in (1, 2):
        out = batch_case(q, args, flush, pk, pk_kind, torch, pkg)
        if rank == 0:
            print(json.dumps({"metric": "batched path DOF-updates/s per RK stage", "impl": "ours", **out}))
    return 0


# affine periodic cubes of B^3 roots of 8^3 cells whose state is far above the
# 129 MB L2: the roofline of the stage kernel where HBM is the bound
OVER_L2 = {
    "cube16p1": ("3d-euler-periodic-cube-16^3-roots-n8-p1", 16, 1),
    "cube16p2": ("3d-euler-periodic-cube-16^3-roots-n8-p2", 16, 2),
}


def over_l2_case(key, args, stream, flush, pk, pk_kind, torch, pkg):
    """FP32 DOF-update rate, stage-kernel roofline (state bytes of the
    affine FP32 form: 8 B per DOF on the first stage, 12 B on the others,
    plus the cell sizes on the last) and the FP32-vs-FP64 difference after a
    few steps from the same nodal values, on one affine periodic cube."""
    name, B, p = OVER_L2[key]
    w = W.periodic_cube_forest(B)
    f32 = pkg.Forest.from_workload(w, p=p, precision=pkg.FP32, cfl=0.1)
    f32.set_stream(stream)
    vals = vortex(f32.quad_points())
    f32.set_state_nodal(vals)
    dof = f32.n_leaves * f32.nv * f32.M * f32.nc
    for _ in range(args.warmup):
        f32.rk_step()
    ms = timed_steps(f32, args.steps, stream, flush, torch)
    value = dof * 3 * args.steps / (ms / 1e3)
    f32.set_timing(True)
    f32.kernel_times()
    timed_steps(f32, args.steps, stream, flush, torch)
    kt = f32.kernel_times()
    f32.set_timing(False)
    stage_ms, stage_n = kt["stage"]
    cells = f32.n_leaves * f32.nc
    alg = dof * 4 * (2 + 3 + 3) / 3.0 + cells * 4 / 3.0
    achieved = alg / (stage_ms / stage_n / 1e3) / 1e9
    # FP32 against FP64 after the same steps from the same nodal values
    nacc = 5
    f32.set_state_nodal(vals)
    f32.set_time(0.0)
    f64 = pkg.Forest.from_workload(w, p=p, precision=pkg.FP64, cfl=0.1)
    f64.set_stream(stream)
    f64.set_state_nodal(vals)
    del vals
    torch.cuda.synchronize()
    t64 = time.perf_counter()
    for _ in range(nacc):
        f64.rk_step()
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t64
    for _ in range(nacc):
        f32.rk_step()
    a = f32.get_state().astype(np.float64)
    b = f64.get_state()
    l2 = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    linf = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    out = {"workload": name, "leaves": f32.n_leaves, "cells": cells, "p": p, "dof": dof,
           "state_bytes_fp32": dof * 4, "value": value, "unit": "DOF-updates/s", "ms_per_step": ms / args.steps,
           "steps": args.steps,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": achieved / pk["hbm_gbs"],
                        "traffic": STAGE_TRAFFIC_BYTES.get((key, f32.tuning()["stage_kernel"])),
                        "traffic_how": TRAFFIC_HOW, "kernel": stage_kernel_name(f32, p),
                        "bytes_per_launch": alg, "avg_launch_us": 1e3 * stage_ms / stage_n,
                        "peak_source": pk_kind,
                        "other_kernels_us_per_step": {"guard": 1e3 * kt["guard"][0] / args.steps,
                                                      "dt": 1e3 * kt["dt"][0] / args.steps}},
           "fp64_value": dof * 3 * nacc / t64,
           "accuracy": {"steps": nacc, "l2_rel_fp32_vs_fp64": l2, "linf_rel_fp32_vs_fp64": linf},
           "tuning": f32.tuning(), "status_word": f32.status_word()}
    f32.close()
    f64.close()
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- serving
# the serving mix: 256 Poisson arrivals at 20/s of periodic cubes of 64-8192
# blocks at p = 1..3, end times drawn in [0.05, 0.5] and scaled by 0.01 in the
# bench line (so that it takes seconds) or by 0.1 with --serve-full
SERVE_MIX = dict(rate=20.0, seed=0, blocks=(64, 8192), degrees=(1, 2, 3), t_end=(0.05, 0.5), t_scale=0.01)


def run_serve(args, sub=False):
    """Continuous batching: Poisson arrivals of independent solves (blast or
    vortex, periodic cubes of 64-8192 blocks, p in 1..3, FP32), each admitted
    by its device footprint, built on a worker thread (forest, initial values
    computed on the GPU at its Gauss points) and advanced in the batch of its
    degree (or on its own stream with --serve-streams).  Reports the
    aggregate DOF-update rate over the whole run and p50/p99 time to
    solution."""
    import torch
    import paper_2502_12620_gb300 as pkg
    from paper_2502_12620_gb300 import serve

    ws, rank, local = dist_env()
    if ws > 1 and not sub:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mix_cfg = dict(SERVE_MIX)
    n_req = args.serve_sub_requests if sub else args.serve_requests
    if args.serve_full and not sub:
        n_req, mix_cfg["t_scale"] = 256, 0.1
    mix = W.serving_mix(n_req, **mix_cfg)
    t_prep = 0.0
    reqs = [serve.Request(m["rid"], m["arrival"], W.periodic_cube_forest(m["B"], n_seg=m["n_seg"]), m["p"],
                          m["t_end"], ("device", serving_device_init(m, torch, dev)), pkg.FP32) for m in mix]
    # warm-up: a small solve of every degree and initial condition, with its
    # initial values computed on the device like the timed requests' (module
    # load, allocator pools, and the first-use compilation of torch's
    # elementwise kernels for this GPU, which on a fresh machine takes seconds)
    warm = []
    for p in SERVE_MIX["degrees"]:
        for kind in ("blast", "vortex"):
            wm = dict(B=2, n_seg=8, p=p, kind=kind, centre=np.array([0.5, 0.5, 0.5]))
            warm.append(serve.Request(-1 - len(warm), 0.0, W.periodic_cube_forest(2), p, 1e-3,
                                      ("device", serving_device_init(wm, torch, dev)), pkg.FP32))
    batched = not args.serve_streams
    serve.Server(device=local, max_active=4, batched=batched).run(warm)
    srv = serve.Server(device=local, max_active=args.serve_active, steps_per_round=8, batched=batched)
    # grow the caching allocator's pool to the serving budget before the timed
    # run (first-time device allocations of many GB would otherwise be timed)
    pkg.reserve_memory(int(0.9 * srv.budget), local)
    serve.reserve_init_memory(int(0.25 * srv.budget), local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as ck:
        t0 = time.perf_counter()
        res = srv.run(reqs, deadline=args.serve_deadline)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    done = [r for r in res if r.status == 0]
    sm = serve.summarize(done or res, wall)
    updates = sum(r.dof * 3 * r.steps for r in res)
    if sub:
        out = {"workload": "serving-mix-periodic-cubes-64-8192-blocks-n8-p1-3-blast-or-vortex",
               "requests": len(res), "value": updates / wall, "unit": "DOF-updates/s",
               "p50_s": sm["p50_s"], "p99_s": sm["p99_s"], "wall_s": wall, "max_active": args.serve_active,
               "mode": "batched: one launch per kernel and stage for the solves of one degree" if batched
               else "one stream and graph per solve",
               "failed": sum(1 for r in res if r.status not in (0, -100, -101)),
               "unfinished_at_deadline": sum(1 for r in res if r.status in (-100, -101)),
               "failed_requests": [dict(rid=m["rid"], B=m["B"], p=m["p"], kind=m["kind"], status=r.status)
                                   for m, r in zip(mix, res) if r.status not in (0, -100, -101)],
               "peak_active": srv.peak_active,
               "mean_queue_s": float(np.mean([r.admitted - r.arrival for r in res])),
               "blocks_max": max(m["B"] ** 3 for m in mix), **{k: list(v) if isinstance(v, tuple) else v for k, v in mix_cfg.items()}}
        if batched:
            # the same requests, one stream and graph per solve (for comparison)
            srv2 = serve.Server(device=local, max_active=args.serve_active, steps_per_round=8, batched=False)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            res2 = srv2.run(reqs, deadline=args.serve_deadline)
            torch.cuda.synchronize()
            wall2 = time.perf_counter() - t1
            sm2 = serve.summarize(res2, wall2)
            out["per_solve_streams"] = {"value": sum(r.dof * 3 * r.steps for r in res2) / wall2,
                                        "p50_s": sm2["p50_s"], "p99_s": sm2["p99_s"], "wall_s": wall2}
        return out
    value, ms = job_throughput(updates, 1e3 * wall, ws)
    if rank != 0:
        return 0
    line = {
        "metric": "serving: aggregate DG DOF-updates/s per RK stage", "value": value, "unit": "DOF-updates/s",
        "n_gpus": ws, "steps": len(res), "warmup": len(warm), "ms_per_step": ms / max(1, len(res)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving-mix-periodic-cubes-64-8192-blocks-n8-p1-3-blast-or-vortex",
                   "requests": len(res), **{k: list(v) if isinstance(v, tuple) else v for k, v in mix_cfg.items()},
                   "max_active": args.serve_active, "hbm_budget_bytes": srv.budget},
        "serve": {"p50_s": sm["p50_s"], "p99_s": sm["p99_s"], "wall_s": wall,
                  "peak_active": srv.peak_active, "peak_bytes": srv.peak_bytes,
                  "failed": sum(1 for r in res if r.status not in (0, -100, -101)),
                  "unfinished_at_deadline": sum(1 for r in res if r.status in (-100, -101)),
                  "failed_requests": [dict(rid=m["rid"], B=m["B"], p=m["p"], kind=m["kind"], status=r.status)
                                      for m, r in zip(mix, res) if r.status not in (0, -100, -101)],
                  "mean_queue_s": float(np.mean([r.admitted - r.arrival for r in res])),
                  "dof_updates": updates,
                  "payload": "initial values computed on the GPU by the build worker (inside the timed run)"},
        "clocks": ck.summary(),
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- dynamic AMR
# every 40 steps the blast front has moved far enough that most regrids change
# the forest; CFL 0.3 / (2p + 1) (0.1 at p = 1, 0.06 at p = 2), 0.02 at p = 3
AMR = dict(B=4, n_seg=8, p=1, refine_above=0.05, coarsen_below=0.01, max_level=4, every=40, limiter=1e-6, r0=0.12)


def run_amr(args, sub=False, p=None, periods=None):
    """Blast on a periodic cube of 4^3 roots with dynamic refinement: the
    device indicator and adaptation (2:1 closure, state moved on the device)
    every `every` steps, the positivity limiter after every stage, FP32.
    The rate counts the DOF updated by each time step (3 stages) over the wall
    time of the whole run, regrids included."""
    import torch
    import paper_2502_12620_gb300 as pkg

    ws, rank, local = dist_env()
    if ws > 1 and not sub:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    cfg = dict(AMR)
    cfg["p"] = p if p is not None else args.amr_p
    cfg["cfl"] = 0.3 / (2 * cfg["p"] + 1) if cfg["p"] < 3 else 0.02
    w = W.periodic_cube_forest(cfg["B"], n_seg=cfg["n_seg"])
    # interface one finest cell wide (three at p = 3: the split of a steeper
    # degree-3 profile leaves children whose means are outside the
    # admissible set, which no limiter can repair)
    width = (1.0 if cfg["p"] < 3 else 3.0) / (cfg["B"] * cfg["n_seg"] * 2 ** (cfg["max_level"] - 1))
    cfg["interface_cells"] = 1 if cfg["p"] < 3 else 3
    # at p = 3 (CFL 0.02) the blast moves a few cells over the run: a wider
    # initial blast gives its interface a leaf count in the 2k-20k range
    cfg["r0"] = AMR["r0"] if cfg["p"] < 3 else 0.2
    ic = lambda x: W.blast(x, (0.5, 0.5, 0.5), r0=cfg["r0"], width=width)
    f = pkg.Forest.from_workload(w, p=cfg["p"], precision=pkg.FP32, device=local, cfl=cfg["cfl"])
    stream = torch.cuda.Stream()
    f.set_stream(stream)
    f.set_limiter(cfg["limiter"])
    # initial refinement: adapt to the projected data until it settles
    for _ in range(cfg["max_level"]):
        f.project(ic)
        f.limit()
        nr, nc = f.adapt(cfg["refine_above"], cfg["coarsen_below"], cfg["max_level"])
        if nr == 0 and nc == 0:
            break
    f.project(ic)
    f.limit()
    f.status_word(reset=True)
    dof_leaf = f.nv * f.M * f.nc
    for _ in range(args.warmup):
        f.rk_step()
    torch.cuda.synchronize()
    steps = (periods if periods is not None else args.steps) * cfg["every"]
    updates = 0
    leaves = []
    regrid_s = 0.0
    regrid_changed_s = 0.0
    changes = 0
    with Clocks(local) as ck:
        t0 = time.perf_counter()
        for i in range(steps):
            L = f.n_leaves
            leaves.append(L)
            f.rk_step()
            updates += L * dof_leaf * 3
            if (i + 1) % cfg["every"] == 0:
                stream.synchronize()  # time the regrid alone
                r0 = time.perf_counter()
                nr, nc = f.adapt(cfg["refine_above"], cfg["coarsen_below"], cfg["max_level"])
                if nr > 0 or nc > 0:
                    f.limit()  # split children of a steep profile can leave the admissible set
                dtr = time.perf_counter() - r0
                regrid_s += dtr
                if nr > 0 or nc > 0:
                    changes += 1
                    regrid_changed_s += dtr
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    status = f.status_word()
    amr = {"leaves_min": min(leaves), "leaves_max": max(leaves), "leaves_end": f.n_leaves,
           "regrids": steps // cfg["every"], "regrids_that_changed_the_forest": changes,
           "regrid_s": regrid_s, "regrid_ms_each": 1e3 * regrid_s / max(1, steps // cfg["every"]),
           "regrid_ms_each_changed": 1e3 * regrid_changed_s / max(1, changes),
           "regrid_ms_each_unchanged": 1e3 * (regrid_s - regrid_changed_s) / max(1, steps // cfg["every"] - changes),
           "wall_s": wall, "status_word": status, "t_end": f.time}
    name = f"3d-blast-periodic-cube-4^3-roots-n8-p{cfg['p']}-adaptive-to-level-4"
    if sub:
        f.close()
        return {"workload": name, "value": updates / wall, "unit": "DOF-updates/s", "steps": steps, **amr, **cfg}
    value, ms = job_throughput(updates, 1e3 * wall, ws)
    if rank != 0:
        return 0
    line = {
        "metric": "dynamic AMR: DG DOF-updates/s per RK stage, regrids included", "value": value,
        "unit": "DOF-updates/s", "n_gpus": ws, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": name, **cfg},
        "amr": amr,
        "clocks": ck.summary(),
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- precision sweep
SWEEP = dict(t_end=0.005, cfl=0.1, vortex_box=20.0, runs=((1, (8, 16, 32)), (2, (8, 16, 32)), (3, (8, 16))))


def _cube_points(B, p, torch, dev, z0=0, z1=None):
    """Gauss points of the affine periodic cube of B^3 roots of 8^3 cells, on
    the device, in the library's nodal order [leaf][cell][point][axis] (leaf
    = root = bx + B by + B^2 bz, cell = i + 8 j + 64 k, point = qx + N qy +
    N^2 qz); with z0, z1 only the roots of the slab z0 <= bz < z1 (leaves
    z0 B^2 .. z1 B^2 - 1)."""
    N = p + 1
    z1 = B if z1 is None else z1
    xg = torch.tensor(np.polynomial.legendre.leggauss(N)[0], dtype=torch.float64, device=dev)
    h = 1.0 / (8 * B)
    b = torch.arange(B, dtype=torch.float64, device=dev)
    c = torch.arange(8, dtype=torch.float64, device=dev)
    # 1D coordinate of (block, cell, point) along one axis
    ax = (b[:, None, None] / B + c[None, :, None] * h + h * (xg[None, None, :] + 1) / 2)  # [B][8][N]
    nz = z1 - z0
    X = ax[None, None, :, None, None, :, None, None, :].expand(nz, B, B, 8, 8, 8, N, N, N)
    Y = ax[None, :, None, None, :, None, None, :, None].expand(nz, B, B, 8, 8, 8, N, N, N)
    Z = ax[z0:z1, None, None, :, None, None, :, None, None].expand(nz, B, B, 8, 8, 8, N, N, N)
    # index order above: [bz][by][bx][k][j][i][qz][qy][qx]
    return torch.stack([X, Y, Z], -1).reshape(nz * B * B, 512, N ** 3, 3)


def _vortex_t(x, t, torch, scale=20.0):
    """The isentropic vortex of the bench mapped into the unit cube from a
    box of `scale` units centred on it (20 in the sweep, so the periodic cut
    of its Gaussian tail, e^-50, sets no error floor; 10 in the serving mix,
    as workloads.serving_initial), translated by the free stream to time t,
    nearest periodic image (as workloads.vortex_exact), on torch tensors:
    conserved variables [..., 5]."""
    beta, gamma, period = 5.0, 1.4, scale
    cx = (scale / 2 + t * scale) % period
    cy = (scale / 2 + t * scale) % period
    X = scale * x[..., 0]
    Y = scale * x[..., 1]
    dx = torch.remainder(X - cx + period / 2, period) - period / 2
    dy = torch.remainder(Y - cy + period / 2, period) - period / 2
    r2 = dx * dx + dy * dy
    e = torch.exp(0.5 * (1.0 - r2))
    u = 1.0 - beta / (2 * math.pi) * e * dy
    v = 1.0 + beta / (2 * math.pi) * e * dx
    w = torch.ones_like(u)
    T = 1.0 - (gamma - 1.0) * beta ** 2 / (8.0 * gamma * math.pi ** 2) * torch.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    pr = rho ** gamma
    E = pr / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, rho * u, rho * v, rho * w, E], -1)


def _blast_t(x, centre, r0, width, torch):
    """workloads.blast on torch tensors: (rho, p) = (8, 10) inside r0, (1, 1)
    outside, at rest, tanh interface of the given width."""
    c = torch.tensor(np.asarray(centre, float), dtype=x.dtype, device=x.device)
    r = torch.sqrt(((x - c) ** 2).sum(-1))
    sh = 0.5 * (1.0 - torch.tanh((r - r0) / width))
    rho = 1.0 + 7.0 * sh
    pr = 1.0 + 9.0 * sh
    z = torch.zeros_like(rho)
    return torch.stack([rho, z, z, z, pr / 0.4], -1)


def serving_device_init(m, torch, dev):
    """Initial values of a serving_mix request computed on the GPU at the
    forest's Gauss points (the same formulas as workloads.serving_initial),
    one slab of roots at a time into the result (about 64 roots a slab), so
    that the formulas' temporaries stay small against the state."""
    def init(f):
        B, N = m["B"], m["p"] + 1
        with torch.no_grad():
            U = torch.empty((B ** 3, 512, N ** 3, 5), dtype=torch.float64, device=dev)
            zs = max(1, 64 // (B * B))
            for z0 in range(0, B, zs):
                z1 = min(B, z0 + zs)
                X = _cube_points(B, m["p"], torch, dev, z0, z1)
                if m["kind"] == "blast":
                    V = _blast_t(X, m["centre"], 0.1, 1.0 / (B * m["n_seg"]), torch)
                else:
                    V = _vortex_t(X, 0.0, torch, scale=10.0)
                U[z0 * B * B:z1 * B * B] = V
                del X, V
            f.set_state_nodal(U)
            del U
    return init


def _to_nodal_t(K, p, torch):
    """Modal [leaf][var][mode][cell] -> values at the Gauss points, on the device."""
    N = p + 1
    x = np.polynomial.legendre.leggauss(N)[0]
    V = torch.tensor([[np.polynomial.legendre.legval(xq, [0] * k + [1]) for k in range(N)] for xq in x],
                     dtype=K.dtype, device=K.device)
    L, nv, M, nc = K.shape
    A = K.reshape(L, nv, N, N, N, nc)  # (k_z, k_y, k_x)
    A = torch.einsum("ak,lvzykc->lvzyac", V, A)
    A = torch.einsum("ak,lvzkxc->lvzaxc", V, A)
    A = torch.einsum("ak,lvkyxc->lvayxc", V, A)
    return A.reshape(L, nv, M, nc)


def run_sweep(args):
    """Accuracy and throughput sweep on periodic cubes of B^3 roots (8^3
    cells each) with the scaled isentropic vortex: FP64, FP32 and the
    compensated FP32 form per (p, B); L2 / Linf error against the exact
    translated vortex (observed order from successive B), FP32 against FP64
    on the same steps, conservation drift, DOF-updates/s."""
    import torch
    import paper_2502_12620_gb300 as pkg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    rows = []
    for p, Bs in SWEEP["runs"]:
        N = p + 1
        wq = torch.tensor(np.polynomial.legendre.leggauss(N)[1], dtype=torch.float64, device=dev)
        W3 = (wq[None, None, :] * wq[None, :, None] * wq[:, None, None]).reshape(-1)  # [q] (qz, qy, qx)
        for B in Bs:
            w = W.periodic_cube_forest(B)
            X = _cube_points(B, p, torch, dev)
            if B == 8:  # the device points are the library's
                h = pkg.Forest.from_workload(w, p=p, device=-1)
                assert np.allclose(h.quad_points(), X.cpu().numpy(), atol=1e-14)
                h.close()
            U0 = _vortex_t(X, 0.0, torch).permute(0, 1, 2, 3).contiguous()  # [leaf][cell][q][v]
            res = {}
            for name, prec in (("fp64", pkg.FP64), ("fp32", pkg.FP32), ("fp32_comp", pkg.FP32_COMP)):
                f = pkg.Forest.from_workload(w, p=p, precision=prec, device=local, cfl=SWEEP["cfl"])
                f.set_stream(stream)
                f.set_state_nodal(U0)
                T0 = f.conserved_totals()
                f.rk_step(t_end=0.0)  # tunes the stage kernel; an increment at t_end is the identity
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                steps = 0
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    while True:
                        f.rk_step(t_end=SWEEP["t_end"])
                        steps += 1
                        if steps % 8 == 0 and f.time >= SWEEP["t_end"] * (1 - 1e-12):
                            break
                    e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1)
                t = f.time
                steps = f.step_count
                T1 = f.conserved_totals()
                K = torch.empty(f.state_shape, dtype=torch.float64 if prec != pkg.FP32 else torch.float32, device=dev)
                f.get_state(K)
                Un = _to_nodal_t(K.double(), p, torch)  # [leaf][var][q][cell]
                del K
                ex = _vortex_t(X, t, torch).permute(0, 3, 2, 1)  # [leaf][var][q][cell]
                d = Un - ex
                l2 = float(torch.sqrt(torch.einsum("q,lvqc->", W3, d * d) / torch.einsum("q,lvqc->", W3, ex * ex)))
                linf = float(d.abs().max() / ex.abs().max())
                del d, ex
                dof = f.n_leaves * f.nv * f.M * f.nc
                res[name] = {"l2_vs_exact": l2, "linf_vs_exact": linf, "steps": steps, "t": t,
                             "dof_updates_per_s": dof * 3 * steps / (ms / 1e3),
                             "conservation_drift": float(np.max(np.abs(T1 - T0)) / np.max(np.abs(T0))),
                             "status_word": f.status_word()}
                if name == "fp64":
                    U64 = Un
                else:
                    dd = Un - U64
                    res[name]["l2_rel_vs_fp64"] = float(torch.linalg.vector_norm(dd) / torch.linalg.vector_norm(U64))
                    res[name]["linf_rel_vs_fp64"] = float(dd.abs().max() / U64.abs().max())
                    del dd
                del Un
                f.close()
                torch.cuda.empty_cache()
            del U64, U0, X
            torch.cuda.empty_cache()
            rows.append({"p": p, "B": B, "leaves": B ** 3, "dof": B ** 3 * 512 * 5 * N ** 3, **res})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    # observed order from successive B (h halves)
    for i in range(1, len(rows)):
        a, b = rows[i - 1], rows[i]
        if a["p"] == b["p"]:
            for name in ("fp64", "fp32", "fp32_comp"):
                b[name]["observed_order"] = math.log2(a[name]["l2_vs_exact"] / b[name]["l2_vs_exact"])
    if rank == 0:
        print(json.dumps({"metric": "precision sweep: error vs exact vortex, FP32 vs FP64, DOF-updates/s",
                          "config": {"workload": "3d-euler-periodic-cube-B^3-roots-n8-isentropic-vortex", **SWEEP},
                          "rows": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="jitter3d", choices=sorted(WORKLOADS))
    ap.add_argument("--quick", action="store_true", help="timed steps only (profiling runs)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_comp"],
                    help="precision of the --quick run")
    ap.add_argument("--serve", action="store_true", help="continuous-batching run instead of the step benchmark")
    ap.add_argument("--amr", action="store_true", help="dynamic-refinement blast run (steps = regrid periods)")
    ap.add_argument("--batch", action="store_true",
                    help="the batched path alone: one batch of three affine cubes at p = 1 and 2")
    ap.add_argument("--sweep", action="store_true", help="accuracy / precision sweep on periodic vortex cubes")
    ap.add_argument("--nonconforming", default="paper", choices=["paper", "mortar"],
                    help="level jumps: the paper's guard-cell scheme (default) or the conservative mortar repair")
    ap.add_argument("--quick-line", action="store_true",
                    help="the step line without the over-L2, serving and AMR sub-objects")
    ap.add_argument("--serve-sub-requests", type=int, default=256)
    ap.add_argument("--amr-sub-periods", type=int, default=30)
    ap.add_argument("--amr-p", type=int, default=1, help="degree of the --amr run")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-full", action="store_true", help="256 requests, end times scaled by 0.1")
    ap.add_argument("--serve-deadline", type=float, default=120.0,
                    help="seconds after which a serving run stops (unfinished requests are reported)")
    ap.add_argument("--serve-streams", action="store_true",
                    help="serve with one stream and graph per solve instead of batches per degree")
    ap.add_argument("--serve-active", type=int, default=8)
    args = ap.parse_args()
    _SEL[0] = args.workload
    _NC[0] = args.nonconforming
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.amr:
        return run_amr(args)
    if args.batch:
        return run_batch(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
