#!/usr/bin/env python3
"""Benchmark of the coupled D3Q19 LB + polymer MD step on GB300.

Workload (default): the paper-shaped translocation box 256 x 128 x 128, wall at
x = 128 with a 5 x 5 pore, one 400-bead chain (seeded self-avoiding walk),
tau = 1, FP32 population storage.  One "step" is one coupled LB step: bead
gather, M = 5 MD substeps, the D3Q19 stream-collide of the whole box and the
spread of the bead impulses.  Metric: MLUPS (all box nodes x steps / s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The same JSON line carries an "ensemble" object (skip with --no-ensemble):
512 independent ragged realisations stepped together with FP16 and with FP32
population storage, against the plain FP32 path stepping one realisation at
a time -- realisation-steps/s and completed realisations/s to a step cap.

For N > 1 the script runs under torch.distributed (one rank per GPU); every
rank steps its own independent realisation (different seed) -- weak scaling
with no collective on the data path; the timed region is bracketed by
barriers and the max over ranks is reported.
"""
from __future__ import annotations

import argparse
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

import seeded_inputs as si  # noqa: E402

BYTES_PER_NODE = {"f32": 152, "f16": 76, "bf16": 76}  # 19 loads + 19 stores


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--streaming", choices=["pull", "aa"], default="pull",
                    help="two-buffer pull streaming or the one-buffer in-place (AA) pattern")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["translocation", "small", "solvent", "poiseuille"],
                    default="translocation")
    ap.add_argument("--box", type=int, default=256, help="edge of the periodic solvent box")
    ap.add_argument("--tau", type=float, default=1.0)
    ap.add_argument("--kT-fluid", type=float, default=0.0,
                    help="temperature of the fluid's thermal source (0: none)")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the batched-ensemble leg")
    ap.add_argument("--ens-count", type=int, default=512)
    ap.add_argument("--ens-steps", type=int, default=400, help="timed ensemble steps")
    ap.add_argument("--ens-cap", type=int, default=2000,
                    help="step cap of the run-to-completion comparison")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of --steps steps each; ms_per_step is their median")
    ap.add_argument("--no-small-box", action="store_true",
                    help="skip the small translocation box (32x16x16, N=20) figure")
    return ap.parse_args()


# parameters of the GPU library that the oracle does not take
GPU_ONLY_KEYS = ("storage", "init_tg_amp", "diag_every", "diag_capacity", "streaming")


def workload(seed: int, storage: str, args=None):
    """Parameters of the timed workload (all inputs seeded and synthetic)."""
    kind = args.workload if args is not None else "translocation"
    if kind == "solvent":
        # periodic box, Taylor-Green start (A = 0.01), body force 1e-6 along x
        p = si.periodic_solvent(args.box, tau=args.tau, g=1e-6)
        p["init_tg_amp"] = 0.01
    elif kind == "poiseuille":
        p = si.poiseuille_channel(256, 128, 128, tau=args.tau, g=1e-6)
    elif kind == "small":
        # 32x16x16 box, 3x3 pore, 20 beads: launch-latency bound, L2-resident
        p = si.small_translocation(seed)
        p["tau"] = args.tau
    else:
        p = si.paper_translocation(seed)
        p["tau"] = args.tau if args is not None else 1.0
    p["storage"] = storage
    if args is not None:
        p["streaming"] = args.streaming
    if args is not None and args.kT_fluid > 0:
        p["kT_fluid"] = args.kT_fluid
    return p


def launches_per_step(p) -> int:
    """Kernels of one coupled step: gather, MD cycle, stream-collide and the
    spread -- in three kernels when the stream-collide moves 480 MB or more
    per step (the fixed-point sum and the owners' records beside it, the
    apply after it), else in two (the apply converts the sums itself); without
    beads the stream-collide alone, plus the step-count kernel with the
    thermal source."""
    if p["n_beads"] > 0:
        nodes = p["nx"] * p["ny"] * p["nz"]
        bytes_per_step = 2 * 19 * nodes * (4 if p.get("storage", "f32") == "f32" else 2)
        return 6 if bytes_per_step >= 480_000_000 else 5
    return 2 if p.get("kT_fluid", 0) > 0 else 1


def workload_name(p) -> str:
    if p.get("kT_fluid", 0) > 0:
        q = dict(p)
        q["kT_fluid"] = 0
        return workload_name(q) + f", fluctuating (kT_fluid={p['kT_fluid']:g})"
    if p["n_beads"] > 0:
        return (f"translocation {p['nx']}x{p['ny']}x{p['nz']}, wall x={p['wall_x']}, "
                f"{p['pore_d']}x{p['pore_d']} pore, N={p['n_beads']} beads, tau={p['tau']}")
    if p.get("y_walls"):
        return f"Poiseuille channel {p['nx']}x{p['ny']}x{p['nz']}, walls y=0,{p['ny'] - 1}, tau={p['tau']}"
    return f"periodic solvent {p['nx']}^3, Taylor-Green A=0.01, g=1e-6, tau={p['tau']}"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_seed(base: int, rank: int) -> int:
    """Seed of the independent realisation a rank steps (weak scaling)."""
    return base + 7919 * rank


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the job is as slow as its
    slowest rank); identity without a process group."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, from before the
    warm-up until the line is printed (every timed region lies inside)."""

    def __init__(self, index: int, period_ms: int = 50):
        self.index, self.period_ms = index, period_ms
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(p, pos, seconds: float):
    """The FP64 oracle, as it stands, on the host cores: full box, as many LB
    steps as fit in about `seconds` (at least one)."""
    import oracle

    cores = oracle.max_threads()
    op = {k: v for k, v in p.items() if k not in GPU_ONLY_KEYS}
    init_u = (si.taylor_green_field(p["nx"], p["ny"], p["nz"], p["init_tg_amp"])
              if p.get("init_tg_amp") else None)
    sim = oracle.OracleSim(op, init_pos=pos, init_u=init_u)
    t0 = time.perf_counter()
    sim.step(1)
    t1 = time.perf_counter()
    per = t1 - t0
    n = max(1, min(50, int(seconds / max(per, 1e-6)) - 1))
    t0 = time.perf_counter()
    sim.step(n)
    dt = time.perf_counter() - t0
    V = p["nx"] * p["ny"] * p["nz"]
    return {"value": V * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n} LB steps of the {p['nx']}x{p['ny']}x{p['nz']} box with "
                      f"{p['n_beads']} beads after 1 warm-up step (FP64, OpenMP)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    p = workload(0, args.storage, args)
    pos = si.saw_chain(p, 0) if p["n_beads"] > 0 else None
    import oracle

    op = {k: v for k, v in p.items() if k not in GPU_ONLY_KEYS}
    init_u = (si.taylor_green_field(p["nx"], p["ny"], p["nz"], p["init_tg_amp"])
              if p.get("init_tg_amp") else None)
    sim = oracle.OracleSim(op, init_pos=pos, init_u=init_u)
    # untimed warm-up: the requested steps, cut short after 30 s (a full-box
    # oracle step takes a few tenths of a second on the host cores)
    warm, tw = 0, time.perf_counter()
    while warm < args.warmup and (warm < 3 or time.perf_counter() - tw < 30.0):
        sim.step(1)
        warm += 1
    budget = 90.0
    t0 = time.perf_counter()
    done = 0
    while done < args.steps and (time.perf_counter() - t0) < budget:
        sim.step(1)
        done += 1
    dt = time.perf_counter() - t0
    V = p["nx"] * p["ny"] * p["nz"]
    value = V * done / dt / 1e6
    line = {
        "impl": "reference", "metric": "coupled D3Q19 MLUPS", "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": done, "warmup": warm,
        "ms_per_step": 1e3 * dt / max(done, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(p), "storage": "f64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": f"{done} of {args.steps} requested steps (time cap {budget:.0f} s) "
                                   "of the full box, FP64 oracle with OpenMP"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_0710_1272_gb300 as lb

    p = workload(shard_seed(0, rank), args.storage, args)
    pos = si.saw_chain(p, shard_seed(0, rank)) if p["n_beads"] > 0 else None
    V = p["nx"] * p["ny"] * p["nz"]
    stream = torch.cuda.Stream()
    clk = ClockSampler(local).__enter__()
    sim = lb.Simulation(p, init_pos=pos, stream=stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # -- warm-up (captures the step graphs) ------------------------------------
    sim.step(args.warmup)
    barrier()

    # -- timed regions: graph replays of the coupled step, `repeats` regions of
    # exactly `steps` steps, each bracketed by barrier + synchronize; the
    # median region is reported
    regions = []
    for _ in range(max(1, args.repeats)):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        barrier()
        regions.append(max_over_ranks([ev0.elapsed_time(ev1)], dist, "cuda")[0])
    ms = statistics.median(regions)
    # one more region of the same length, captured as one graph with event
    # nodes around every stream-collide on its own stream
    sim.set_kernel_timing(True)
    barrier()
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    sim.step(args.steps)
    ev3.record(stream)
    barrier()
    lb_ms, lb_n = sim.lb_kernel_time()
    sim.set_kernel_timing(False)
    ms_direct = max_over_ranks([ev2.elapsed_time(ev3)], dist, "cuda")[0]
    st = sim.status()

    # -- end to end through the public API with host buffers ------------------
    # Every step: lbmd_step_read_async -- one step and the read-out of its
    # status word, positions and velocities into page-locked host memory
    # (double-buffered); the host waits for step k's block after step k+1 is
    # enqueued and checks it.
    e2e_steps = args.e2e_steps
    N = p["n_beads"]
    nbytes = lb.bead_block_bytes(N)
    blocks = [torch.empty(nbytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    evs = [torch.cuda.Event(), torch.cuda.Event()]
    step0 = st["step"]

    def consume(k):
        evs[k % 2].synchronize()
        status, pos_k, _ = lb.decode_bead_block(blocks[k % 2].numpy(), N)
        assert status["step"] == step0 + k + 1 and np.isfinite(pos_k).all()

    # the step-and-read-out graphs of both step parities exist before the
    # timed loop
    for k in range(2):
        lb.lbmd_step_read_async(sim.ctx, blocks[k].data_ptr(), nbytes)
    step0 += 2
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        lb.lbmd_step_read_async(sim.ctx, blocks[k % 2].data_ptr(), nbytes)
        evs[k % 2].record(stream)
        if k > 0:
            consume(k - 1)
    if e2e_steps > 0:
        consume(e2e_steps - 1)
    barrier()
    e2e_s = max_over_ranks([time.perf_counter() - t0], dist, "cuda")[0]

    del sim
    torch.cuda.empty_cache()
    small_out = None
    if not args.no_small_box and args.workload == "translocation":
        small_out = small_box_leg(args, lb, torch, dist, rank, world)
    ens_out = None if args.no_ensemble else ensemble_leg(args, lb, torch, dist, rank, world)
    clk.__exit__(None, None, None)

    if rank != 0:
        dist.destroy_process_group()
        return 0

    value = world * V * args.steps / (ms / 1e3) / 1e6
    peak, peak_kind = measured_peak_hbm()
    solid = si.solid_mask(p)
    fluid = int(V - solid.sum())
    bytes_per_launch = BYTES_PER_NODE[args.storage] * fluid
    lb_avg_s = lb_ms / 1e3 / max(lb_n, 1)
    achieved = bytes_per_launch / lb_avg_s / 1e9
    if args.streaming == "aa":
        kernel = "k_aa_stream_collide"
    elif args.storage != "f32" and p["nx"] % 2 == 0:
        kernel = "k_stream_collide_pair"  # 16-bit storage, two x-adjacent nodes per thread
    else:
        kernel = "k_stream_collide"
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "lb_stream_collide_traffic.json")
    if os.path.exists(tpath):
        try:
            with open(tpath) as f:
                records = json.load(f)["records"]
            rev = kernel_rev(kernel)
            for tj in records:
                if (tj["kernel"], tj["storage"], tj["workload"], tj["kernel_rev"]) == \
                        (kernel, args.storage, workload_name(p), rev):
                    traffic = tj["bytes_per_launch"]
        except (OSError, ValueError, KeyError, TypeError):
            traffic = None
    clocks = clk.summary()
    line = {
        "metric": "coupled D3Q19 MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "timing": {"repeats": len(regions), "statistic": "median of the timed regions",
                   "ms_per_step_each": [r / args.steps for r in regions]},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.storage, "data": "synthetic",
        "config": {"workload": workload_name(p), "storage": args.storage,
                   "streaming": args.streaming,
                   "seed": shard_seed(0, rank), "parallelism":
                   "independent realisation per GPU" if world > 1 else "1 GPU",
                   "l2": (f"no flush: populations {2 * BYTES_PER_NODE[args.storage] * V / 2 / 1e6:.1f} "
                          "MB read+written per step > 129 MB L2" if BYTES_PER_NODE[args.storage] * V > 129e6
                          else "fits in L2: not an HBM figure")},
        "coupled_steps_per_s": world * args.steps / (ms / 1e3),
        "value_with_kernel_events": world * V * args.steps / (ms_direct / 1e3) / 1e6,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kernel, "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "avg_launch_ms": lb_avg_s * 1e3, "launches_timed": lb_n},
        "e2e": {"value": world * V * e2e_steps / e2e_s / 1e6, "unit": "MLUPS",
                # unwrapped positions and velocities (3N doubles each) and the
                # 24-byte status word
                "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": nbytes,
                "api": ("lbmd_step_read_async (one graph launch of the step and the kernel that "
                        "writes its bead block into a pinned host block, double-buffered; "
                        "the host waits for and checks step k's block after enqueuing step k+1); "
                        "the state stays resident on the GPU between steps, so no host-to-device "
                        "copy per step; the field read-outs (lbmd_read_fields, "
                        "lbmd_read_populations) are not part of the loop")},
        "gpu_launches": launches_per_step(p) * args.steps,
        "clocks": clocks,
        "status": st,
    }
    if small_out is not None:
        line["small_box"] = small_out
    if ens_out is not None:
        line["ensemble"] = ens_out
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, pos, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def small_box_leg(args, lb, torch, dist, rank, world):
    """The small translocation box (32x16x16, 3x3 pore, N = 20, tau = 1,
    same bead parameters): launch- and latency-bound, L2-resident.  Graph
    replays of `steps` coupled steps, median of `repeats` regions."""
    p = si.small_translocation(shard_seed(0, rank))
    p["storage"] = args.storage
    p["streaming"] = args.streaming
    sim = lb.Simulation(p, init_pos=si.saw_chain(p, shard_seed(0, rank)))
    sim.step(max(args.warmup, 3))
    regions = []
    for _ in range(max(1, args.repeats)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(sim.stream)
        sim.step(args.steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        regions.append(max_over_ranks([e0.elapsed_time(e1)], dist, "cuda")[0])
    del sim
    ms = statistics.median(regions) / args.steps
    V = p["nx"] * p["ny"] * p["nz"]
    return {"workload": workload_name(p), "coupled_steps_per_s": world * 1e3 / ms,
            "ms_per_step": ms, "mlups": world * V / ms / 1e3, "steps": args.steps,
            "repeats": len(regions), "l2": "fits in L2 (1.2 MB of populations): not an HBM figure"}


def ensemble_leg(args, lb, torch, dist, rank, world):
    """Batched ragged ensemble (independent translocation realisations, N from
    {20, 50, 100, 200, 400}, boxes (4 N^0.6, 2 N^0.6, 2 N^0.6) rounded to 16,
    pore 3 or 5, own seed and self-avoiding start each) stepped in one set of
    launches per step, FP16 and FP32 storage, against the plain FP32 path that
    steps one realisation at a time.

    Throughput: `ens_steps` timed steps of every realisation (CUDA events).
    Completion: every realisation run until it translocates or reaches the
    step cap `ens_cap` (wall clock, host checks every 256 steps included); the
    plain path runs one realisation of each (N, pore) class to the same end
    and is scaled by the class counts."""
    members, starts = si.ragged_ensemble(args.ens_count, seed=shard_seed(0, rank))
    cells = sum(m["nx"] * m["ny"] * m["nz"] for m in members)
    fluid = sum(m["nx"] * m["ny"] * m["nz"] - int(si.solid_mask(m).sum()) for m in members)
    count = len(members)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    out = {"workload": (f"{count} ragged realisations, N in {{20,50,100,200,400}}, "
                        f"{cells} nodes, eps={members[0]['lj_eps']}"),
           "cells": cells}
    peak, _ = measured_peak_hbm()
    for storage in ("f16", "f32"):
        ens = lb.Ensemble([dict(m, storage=storage) for m in members], starts)
        ens.autotune(2)
        tuning = ens.tuning()
        ens.step(16)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ens.step(args.ens_steps)
        e1.record()
        barrier()
        ms = max_over_ranks([e0.elapsed_time(e1)], dist, "cuda")[0]
        ens.set_kernel_timing(True)
        ens.step(20)
        kt = ens.kernel_times()
        ens.set_kernel_timing(False)
        lb_ms = kt["lb_ms"] / max(kt["steps"], 1)
        achieved = BYTES_PER_NODE[storage] * fluid / (lb_ms / 1e3) / 1e9
        del ens
        torch.cuda.empty_cache()
        # run to completion (translocation or the cap) from a fresh start
        ens = lb.Ensemble([dict(m, storage=storage) for m in members], starts)
        ens.autotune(2)
        barrier()
        t0 = time.perf_counter()
        ens.run(args.ens_cap, check_every=256)
        barrier()
        wall = max_over_ranks([time.perf_counter() - t0], dist, "cuda")[0]
        res = ens.results()
        del ens
        torch.cuda.empty_cache()
        out[storage] = {
            "realisation_steps_per_s": world * count * args.ens_steps / (ms / 1e3),
            "mlups": world * cells * args.ens_steps / (ms / 1e3) / 1e6,
            "ms_per_step": ms / args.ens_steps,
            "stream_collide": {"avg_launch_ms": lb_ms, "achieved_gbs": achieved, "frac": achieved / peak,
                               "tuning": tuning},
            "completed_per_s": world * count / wall, "completion_wall_s": wall,
            "translocated": int((res["state"] == 1).sum()),
        }
    # plain FP32 path, one realisation at a time: one per (N, pore) class
    classes = {}
    for k, m in enumerate(members):
        classes.setdefault((m["n_beads"], m["pore_d"]), []).append(k)
    seq_steps_s, seq_total = 0.0, 0.0
    for (n, d), ks in sorted(classes.items()):
        k = ks[0]
        sim = lb.Simulation(dict(members[k], storage="f32"), init_pos=starts[k])
        sim.step(8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = 8
        while done < args.ens_cap and sim.status()["state"] == 0:
            sim.step(min(256, args.ens_cap - done))
            done = min(args.ens_cap, done + 256)
        torch.cuda.synchronize()
        per_step = (time.perf_counter() - t0) / max(done - 8, 1)
        seq_total += len(ks) * per_step * done
        seq_steps_s += len(ks) * per_step
        del sim
    out["plain_f32_sequential"] = {
        "realisation_steps_per_s": count / seq_steps_s,
        "completed_per_s": count / seq_total,
        "sample": f"one realisation per (N, pore) class ({len(classes)} classes) run to "
                  f"translocation or {args.ens_cap} steps, scaled by the class counts",
    }
    out["cap_steps"] = args.ens_cap
    out["f16_vs_plain_f32_completed"] = out["f16"]["completed_per_s"] / out["plain_f32_sequential"]["completed_per_s"]
    out["f16_vs_f32_ensemble_completed"] = out["f16"]["completed_per_s"] / out["f32"]["completed_per_s"]
    return out


KERNEL_SOURCES = {
    "k_stream_collide": ("lb_kernels.cu", "lb_collide.cuh", "lb_pull.cuh", "lbmd_common.cuh",
                         "lbmd_internal.h"),
    "k_stream_collide_pair": ("lb_kernels.cu", "lb_collide.cuh", "lb_pull.cuh", "lbmd_common.cuh",
                              "lbmd_internal.h"),
    "k_aa_stream_collide": ("lb_aa.cu", "lb_aa.cuh", "lb_collide.cuh", "lb_pull.cuh",
                            "lbmd_common.cuh", "lbmd_internal.h"),
}


def kernel_rev(kernel: str = "k_stream_collide") -> str:
    """Hash of a stream-collide kernel's sources: a stored DRAM-traffic figure
    is only reported while the kernel it was measured on is unchanged."""
    import hashlib

    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_0710_1272_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
