#!/usr/bin/env python
"""Benchmark of the batched hierarchical products Q~v and Q~^T w on GB300.

A step is one pass of the whole path over a batch of synthetic rigid bodies
(all inputs resident in HBM): the bisection tree (Sec. 2.1), the FP64 node
transforms (Sec. 3, Eq. 3.5), Q~v (Algorithm 2) and Q~^T w (Algorithm 3)
in FP32, through the C ABI (zq_pipeline); the timed steps are direct
launches with the dominant kernel bracketed by CUDA events, and the same step
captured in a CUDA graph is timed beside it.  Default workload: 2000 jittered sphere shells, n_j log-uniform in
[50, 5000] (radius 0.1 sqrt(n_j), jitter 2.5% of the radius, centres uniform
in a 100^3 box).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own batch (seed = rank): weak scaling, no
data-path collective; the barrier and the max over ranks are the only
communication.  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = ("beads/s for batched Q̃v+Q̃ᵀv (FP32 vs FP64 GPU) at stated error; "
          "% HBM peak")
FP64_PEAK_NOMINAL = 1.25e12  # FP64 flop/s, GB300 nominal (FP64 FMA counted as 2 flops)
# The double-single build runs its FP64-class arithmetic on the FP32 pipes.
# Its ALU ceiling: 152 SMs x 128 FP32 lanes x 2070 MHz = 4.03e13 FP32
# operations/s, divided by the FP32 operations one FP64-equivalent flop
# costs in zq_real.cuh: a dd add 20, a dd multiply 7, so a multiply-add
# a*b + c costs 27 for its 2 flops (13.5 per flop; the Householder steps
# are multiply-add chains).
DD_OPS_PER_FLOP = 13.5
DD_PEAK_DERIVED = 152 * 128 * 2.07e9 / DD_OPS_PER_FLOP


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["shells2000", "ellipsoid"], default="shells2000")
    ap.add_argument("--bodies", type=int, default=2000,
                    help="bodies of the shell workload (smaller values: profiling captures)")
    ap.add_argument("--cut", type=int, default=0,
                    help="level cut (performance only); 0: chosen by the autotuner on this workload")
    ap.add_argument("--schedule", choices=["auto", "levels", "fused"], default="auto",
                    help="step schedule after the tree (performance only): level launches, the fused per-body "
                         "launch, or auto (the autotuner times both, with every level cut)")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of the autotuner's picks per workload shape (read and updated)")
    ap.add_argument("--build", choices=["dd", "fp64"], default="dd",
                    help="node-transform arithmetic: double-single on FP32 pipes or native FP64")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip FP64 / apply-only / e2e / CPU legs")
    ap.add_argument("--extras", default="all",
                    help="comma-separated subset of the extra legs: error, build_other, fp64_step, apply, qgen, "
                         "e2e, multirhs, ellipsoid, bd_loop, cpu (default all)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-phases", action="store_true",
                    help="skip the per-kernel timing pass (the dominant kernel is then build_level)")
    return ap.parse_args()


# ------------------------------------------------------------------ setup


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch

            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, x: float, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, x: float, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def make_workload(name: str, seed: int, bodies: int = 2000):
    from paper_1708_08427_gb300 import workloads as W

    if name == "shells2000":
        bt = W.shell_batch(m=bodies, nmin=50, nmax=5000, seed=seed)
        desc = (f"batched jittered sphere shells: m={bodies}, n_j log-uniform [50,5000], radius "
                "0.1*sqrt(n_j), jitter 0.025*radius, centres U[0,100]^3")
    else:
        bt = W.ellipsoid_body(n=1 << 20, seed=seed)
        desc = "one ellipsoid body, n=2^20, semi-axes (3,2,1)*sqrt(n)/100, radial jitter N(0,0.01^2)"
    return bt, desc


# --------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ work model


def node_census(ctx):
    """Counts of internal nodes by transform size k (3, 6, 9)."""
    t = ctx.get_tree()
    internal = (t["left"] >= 0).astype(np.int64) + (t["right"] >= 0).astype(np.int64)
    return {3: int((internal == 0).sum()), 6: int((internal == 1).sum()), 9: int((internal == 2).sum())}


# FP64 flops of one node transform (sqrt and division count 1, FMA 2), as
# counted from the algorithm: geometry (1/n, centroid, offset,
# sqrt(n_x/n), sqrt(n_y/n), sqrt(n_x n_y/n)) 23; Case I closed form 32;
# Householder LQ restricted to the nonzero pattern of [T22_x | T22_y | K]:
# k = 6: K 3, ||M||_F 22, reflectors 29 + 30 + 16; k = 9: K 3, ||M||_F 32,
# reflectors 40 + 44 + 25.
BUILD_FLOPS = {3: 23 + 32, 6: 23 + 3 + 22 + 29 + 30 + 16, 9: 23 + 3 + 32 + 40 + 44 + 25}


def build_flops(k: int) -> int:
    return BUILD_FLOPS[k]


# words of the node record a sweep needs: Case I alpha, beta, G (11);
# k = 6: alpha, beta, 3 tau, 2 + 3 + 3 reflector entries (13); k = 9:
# alpha, beta, 3 tau, 3 + 5 + 6 (19)
RECORD_FLOATS = {3: 11, 6: 13, 9: 19}


def sweep_bytes(census, N, R, es=4, gather=True) -> int:
    """Algorithmic DRAM bytes of one sweep (up or down): the bead-vector
    planes (3N) and residues (R) once, each node record once (by k), the
    node structure (two child codes and the residue offset, 12 B) and, for
    vectors in the caller's order (gather), the sorted-position -> bead map
    (4 B per bead).  The Info-/Velocity-sets that the implementation passes
    between heights through global memory are not counted (the method needs
    them only on chip)."""
    rec = sum(census[k] * RECORD_FLOATS[k] * es for k in census)
    nodes = sum(census.values())
    return es * (3 * N + R) + rec + 12 * nodes + (4 * N if gather else 0)


def kernel_work(name, census, N, R, m, es):
    """(bound, algorithmic amount per launch, unit)."""
    if name in ("build", "fused"):  # every node's transform (the fused step also runs both sweeps)
        return "alu", sum(census[k] * build_flops(k) for k in census), "flop"
    if name in ("up_seg", "down_seg"):  # the step's sweeps see tree-ordered planes (no gather)
        return "hbm", sweep_bytes(census, N, R, es, gather=False), "B"
    if name == "sort_small":
        return "hbm", 8 * N + 8 * N + 4 * N, "B"
    if name == "bottom_up":
        nodes = N - m
        return "hbm", N * 1 + nodes * (4 * 6 + 1), "B"
    return "hbm", 24 * N, "B"


def sources_sha256(paths) -> str:
    """sha256 over the concatenated contents of the files a kernel is built
    from (paths relative to the repository root)."""
    h = hashlib.sha256()
    for rel in paths:
        h.update((ROOT / rel).read_bytes())
    return h.hexdigest()


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (else None)."""
    f = ROOT / "profiles" / "traffic.json"
    if not f.exists():
        return None
    try:
        d = json.loads(f.read_text())
        e = d.get(kernel)
        if not e:
            return None
        if sources_sha256(e.get("sources") or [e["source"]]) != e["sha256"]:
            return None
        return float(e["dram_bytes_per_launch"]) * float(e.get("scale", 1.0))
    except Exception:
        return None


# ------------------------------------------------------------ our arm


def run_ours(args, world, rank, local):
    import torch

    from paper_1708_08427_gb300 import zq

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    bt, desc = make_workload(args.workload, seed=rank, bodies=args.bodies)
    N, m, R = bt.N, bt.m, bt.n_residues
    stream = torch.cuda.Stream(device=dev)
    rng = np.random.default_rng(1000 + rank)
    with torch.cuda.stream(stream):
        x, y, z = (torch.from_numpy(a).to(dev) for a in (bt.x, bt.y, bt.z))
        v = torch.from_numpy(rng.standard_normal((3, N))).to(dev, torch.float32)
        w = torch.from_numpy(rng.standard_normal(R)).to(dev, torch.float32)
        qv = torch.empty(R, dtype=torch.float32, device=dev)
        qtw = torch.empty((3, N), dtype=torch.float32, device=dev)
        flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream.synchronize()
    _XYZ[id(bt)] = (x, y, z)
    ctx = zq.Context(local, stream=stream)
    ctx.set_build_arith(args.build)
    tuned, from_cache = None, False
    if args.schedule == "auto" or args.cut == 0:  # chosen by timing the step itself
        from paper_1708_08427_gb300.tune import CANDIDATES, tune_level_cut, tune_step

        if args.schedule == "levels":
            args.cut, tuned = tune_level_cut(ctx, bt.off, x, y, z, v, qv, w, qtw, graph=not args.no_graph)
        elif args.schedule == "fused":
            args.cut = args.cut or 15
        else:
            cands = CANDIDATES if args.cut == 0 else (("levels", args.cut), ("fused", 0))
            (args.schedule, cut), tuned, from_cache = tune_step(
                ctx, bt.off, x, y, z, v, qv, w, qtw, candidates=cands, graph=not args.no_graph,
                cache=args.tune_cache, key_extra={"arith": args.build})
            args.cut = cut or args.cut or 15
    ctx.set_step_schedule(args.schedule)

    # the step is one zq_pipeline call; with graphs on, the library captures
    # it once and replays it (ZQ_GRAPH), the timing events included
    def step(graph=not args.no_graph):
        ctx.pipeline(bt.off, x, y, z, v, qv, w, qtw, level_cut=args.cut, graph=graph)

    def step_direct():
        step(graph=False)

    for _ in range(max(args.warmup, 1)):
        step()
    ctx.sync()
    census = node_census(ctx)

    # --- per-kernel time of one step (measurement hook), picks the dominant kernel
    names = (["small_tree", "aabb", "keys", "sort_radix", "lcp", "bottom_up", "scan", "fused"]
             if args.schedule == "fused" else
             ["small_tree", "aabb", "keys", "sort_radix", "lcp", "bottom_up", "scan", "segments",
              "schedule", "build", "build_level", "build_tail", "to_tree", "up_seg_early", "up_seg", "up_top", "down_top",
              "down_seg", "from_tree"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e1.record(stream)
    phases = {}
    for nm in ([] if args.no_phases else names):
        ctx.time_kernel(nm, e0, e1)
        tot = 0.0
        e0.record(stream)
        e1.record(stream)
        stream.synchronize()
        reps = 3
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            step()
            stream.synchronize()
            tot += e0.elapsed_time(e1)
        ctx.time_kernel(None)
        phases[nm] = tot / reps
    # candidates: the transform build as a whole (Case I kernel, level
    # launches and the part above the cut), each sweep, the tree, the schedules
    dominant = max(("build", "up_seg", "down_seg", "small_tree", "schedule", "segments", "fused"),
                   key=lambda k: phases.get(k, 0.0)) if phases else ("fused" if args.schedule == "fused" else "build")

    # --- the dominant kernel is bracketed by events in every timed step
    # (external event records: in a replayed step they are graph nodes)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    k1.record(stream)
    stream.synchronize()
    ctx.time_kernel(dominant, k0, k1)
    before = ctx.launch_count()
    step()
    stream.synchronize()
    launches_per_step = ctx.launch_count() - before
    ctx.sync()

    def run_step():
        step()

    for _ in range(args.warmup):
        run_step()
    stream.synchronize()

    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms, kern_ms = [], []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()                    # L2 flush, outside the events
        s0.record(stream)
        run_step()
        s1.record(stream)
        stream.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        kern_ms.append(k0.elapsed_time(k1))
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ctx.time_kernel(None)
    ctx.sync()

    t_dev = sum(step_ms) / 1e3
    t_max = max_over_ranks(world, t_dev, dev)
    beads_total = sum_over_ranks(world, float(N) * args.steps, dev)
    value = beads_total / t_max
    ms_per_step = 1e3 * t_max / args.steps

    bound, work, unit = kernel_work(dominant, census, N, R, m, 4)
    kavg = statistics.mean(kern_ms) / 1e3
    if bound == "alu" and args.build == "dd":
        achieved, peak, runit = work / kavg / 1e12, DD_PEAK_DERIVED / 1e12, "TFLOP/s"
        peak_note = ("derived: FP32 lane rate 152 x 128 x 2070 MHz / 13.5 FP32 ops per FP64-equivalent "
                     "flop of the double-single arithmetic")
    elif bound == "alu":
        achieved, peak, runit = work / kavg / 1e12, FP64_PEAK_NOMINAL / 1e12, "TFLOP/s"
        peak_note = "FP64 nominal 1.25 TFLOP/s (GB300 spec table)"
    else:
        peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        achieved, peak, runit = work / kavg / 1e9, hbm, "GB/s"
        peak_note = "of measured" if peaks else "of fallback"
    traffic = traffic_for(dominant)
    roofline = {"kernel": dominant, "bound": bound, "achieved": achieved, "peak": peak, "unit": runit,
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_note,
                "work_per_launch": work, "work_unit": unit, "kernel_ms": 1e3 * kavg}

    out = {
        "metric": METRIC, "value": value, "unit": "beads/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 sweeps; transforms " + ("double-single (2 x f32, ~48-bit)" if args.build == "dd" else "f64"),
        "data": "synthetic (seeded numpy generators; no dataset)",
        "config": {"workload": desc, "m": m, "N": N, "residues": R, "schedule": args.schedule,
                   "level_cut": args.cut, "schedule_tuning_ms": tuned, "tuning_from_cache": from_cache,
                   "graph": not args.no_graph, "prec": "fp32", "build": args.build,
                   "step": ("tree + transforms (" + ("double-single" if args.build == "dd" else "FP64")
                            + ") + Q~v + Q~^T w, one C-ABI call (zq_pipeline)"),
                   "l2": "512 MB buffer written before every step, outside the step events",
                   "wall_s_timed_region": wall},
        "roofline": roofline, "clocks": clk, "gpu_launches": launches_per_step * args.steps,
        "phases_ms": phases,
    }

    # the outputs of the last timed step against the FP64 oracle (rank 0):
    # the error the metric is stated at
    legs = set() if args.no_extras else (
        {"error", "build_other", "fp64_step", "apply", "qgen", "e2e", "multirhs", "ellipsoid", "bd_loop", "cpu"}
        if args.extras == "all" else set(args.extras.split(",")))
    if rank == 0 and "error" in legs:
        stream.synchronize()
        out["config"]["stated_error"] = step_error(bt, v, w, qv, qtw)

    # each sweep of the step against HBM (per-kernel events, algorithmic bytes)
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sweeps = {}
    for nm in ("up_seg", "down_seg"):
        if phases.get(nm):
            # the upward sweep's segments run in two launches (those at or
            # below the level cut beside the build, the rest after it)
            ms = phases[nm] + (phases.get("up_seg_early", 0.0) if nm == "up_seg" else 0.0)
            byt = sweep_bytes(census, N, R, 4, gather=False)
            sweeps[nm] = {"ms": ms, "algorithmic_bytes": byt, "hbm_frac": byt / (ms / 1e3) / 1e9 / hbm_peak}
    roofline["sweeps_in_step"] = sweeps

    if not args.no_graph:
        # the same step without the library's graph, captured by torch instead
        out["graph_replay"] = timed(args, step_direct, stream, flush, world, dev, N, graph=True)
        out["direct_launches"] = timed(args, step_direct, stream, flush, world, dev, N, graph=False)
        # the library's graph without the kernel-timing event nodes of the timed steps
        out["library_graph_untimed"] = timed(args, step, stream, flush, world, dev, N, graph=False)
    if "build_other" in legs:
        other = "fp64" if args.build == "dd" else "dd"
        ctx.set_build_arith(other)
        out[f"build_{other}_step"] = timed(args, step_direct, stream, flush, world, dev, N,
                                           graph=not args.no_graph)
        ctx.set_build_arith(args.build)
    if "fp64_step" in legs:
        out["fp64_step"] = fp64_step(args, ctx, bt, stream, flush, rng, world, dev)
    if "apply" in legs:
        out["apply"] = apply_only(args, ctx, bt, stream, flush, census, v, w, qv, qtw, world, dev)
    if "qgen" in legs:
        out["qgen"] = qgen_bench(args, ctx, bt, stream, flush, world, dev)
    if "e2e" in legs:
        out["e2e"] = e2e(args, ctx, bt, stream, world, dev)
    if "multirhs" in legs:
        out["multirhs"] = multirhs(args, stream, flush, world, dev, rank)
    if "ellipsoid" in legs and args.workload != "ellipsoid":
        out["ellipsoid_2e20"] = ellipsoid_leg(args, stream, flush, world, dev, rank)
    if "bd_loop" in legs:
        out["bd_loop"] = bd_loop(args, stream, flush, world, dev, rank)
        out["bd_loop_rotation_reuse"] = bd_loop(args, stream, flush, world, dev, rank, reuse=True)
    if rank == 0 and "cpu" in legs:
        out["cpu_baseline"] = cpu_baseline(bt, args.cpu_seconds)
    ctx.close()
    # FP32 against the plain FP64 GPU form, in the kept part of the line
    cmp = {"fp32_step_ms": ms_per_step}
    if "fp64_step" in out:
        cmp["fp64_sweeps_step_ms"] = out["fp64_step"]["ms_per_step"]
        cmp["speedup_vs_fp64_sweeps"] = out["fp64_step"]["ms_per_step"] / ms_per_step
    other = "fp64" if args.build == "dd" else "dd"
    if f"build_{other}_step" in out:
        cmp[f"build_{other}_step_ms"] = out[f"build_{other}_step"]["ms_per_step"]
    if "apply" in out:
        for nm in ("fp32", "fp32_tree_order", "fp64"):
            cmp[f"apply_pair_{nm}_ms"] = out["apply"][nm]["ms_per_step"]
            cmp[f"apply_pair_{nm}_hbm_frac"] = out["apply"][nm]["hbm_frac"]
    out["config"]["fp32_vs_fp64_gpu"] = cmp
    # a short summary as the line's last key (the end of the line is what
    # log tails keep)
    se = out["config"].get("stated_error", {})
    out["summary"] = {"ms": round(ms_per_step, 4), "err_elem": se.get("worst_element"),
                      "err_norm": se.get("worst_norm"),
                      "fp64_ms": round(cmp["fp64_sweeps_step_ms"], 4) if "fp64_sweeps_step_ms" in cmp else None,
                      "up_frac": round(sweeps["up_seg"]["hbm_frac"], 3) if "up_seg" in sweeps else None,
                      "down_frac": round(sweeps["down_seg"]["hbm_frac"], 3) if "down_seg" in sweeps else None,
                      "pair_tree_frac": round(cmp["apply_pair_fp32_tree_order_hbm_frac"], 3)
                      if "apply_pair_fp32_tree_order_hbm_frac" in cmp else None,
                      "ellipsoid_ms": round(out["ellipsoid_2e20"]["ms_per_step"], 4) if "ellipsoid_2e20" in out else None}
    return out


def step_error(bt, v, w, qv, qtw):
    """Every output of the timed step (FP32 Q~v and Q~^T w of the whole
    batch) against the FP64 oracle on the same (FP32-rounded) inputs: per
    body the relative 2-norm error and the worst element error relative to
    the body's largest |element|; the worst of each over all bodies."""
    import oracle
    from paper_1708_08427_gb300 import workloads as W

    vr = v.double().cpu().numpy()
    wr = w.double().cpu().numpy()
    got_q = qv.double().cpu().numpy()
    got_qt = W.interleave(*qtw.double().cpu().numpy())
    t0 = time.perf_counter()
    rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, W.interleave(*vr), wr)
    dt = time.perf_counter() - t0
    worst = {"qv_norm": 0.0, "qv_element": 0.0, "qtw_norm": 0.0, "qtw_element": 0.0}
    ro = 0
    for j in range(bt.m):
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        for key, g, r in (("qv", got_q[ro:ro + 3 * n - 6], rq[ro:ro + 3 * n - 6]),
                          ("qtw", got_qt[3 * o:3 * (o + n)], rqt[3 * o:3 * (o + n)])):
            worst[key + "_norm"] = max(worst[key + "_norm"], float(np.linalg.norm(g - r) / np.linalg.norm(r)))
            worst[key + "_element"] = max(worst[key + "_element"], float(np.abs(g - r).max() / np.abs(r).max()))
        ro += 3 * n - 6
    return {"against": "FP64 oracle, every body of the timed batch (last timed step's outputs)",
            "bodies": bt.m, "tolerance": 1e-5, **worst,
            "worst_norm": max(worst["qv_norm"], worst["qtw_norm"]),
            "worst_element": max(worst["qv_element"], worst["qtw_element"]), "oracle_s": dt}


def fp64_step(args, ctx, bt, stream, flush, rng, world, dev):
    """The plain FP64 GPU form: the same step with FP64 sweeps."""
    import torch

    N, R = bt.N, bt.n_residues
    v = torch.from_numpy(rng.standard_normal((3, N))).to(dev)
    w = torch.from_numpy(rng.standard_normal(R)).to(dev)
    qv = torch.empty(R, dtype=torch.float64, device=dev)
    qtw = torch.empty((3, N), dtype=torch.float64, device=dev)
    stream.synchronize()

    def step():
        ctx.pipeline(bt.off, *xyz_of(ctx, bt, dev), v, qv, w, qtw, level_cut=args.cut)

    return timed(args, step, stream, flush, world, dev, N, graph=not args.no_graph)


_XYZ = {}


def xyz_of(ctx, bt, dev):
    import torch

    key = id(bt)
    if key not in _XYZ:
        _XYZ[key] = tuple(torch.from_numpy(a).to(dev) for a in (bt.x, bt.y, bt.z))
    return _XYZ[key]


def timed(args, fn, stream, flush, world, dev, N, graph=True, steps=None):
    import torch

    steps = steps or max(3, min(args.steps, 10))
    for _ in range(2):
        fn()
    stream.synchronize()
    g = None
    if graph:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        stream.synchronize()
    run = (lambda: g.replay()) if g is not None else fn
    for _ in range(2):
        with torch.cuda.stream(stream):
            run()
    stream.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        s0.record(stream)
        with torch.cuda.stream(stream):
            run()
        s1.record(stream)
        stream.synchronize()
        ms.append(s0.elapsed_time(s1))
    t = max_over_ranks(world, sum(ms) / 1e3, dev)
    tot = sum_over_ranks(world, float(N) * steps, dev)
    return {"value": tot / t, "unit": "beads/s", "ms_per_step": 1e3 * t / steps, "steps": steps}


def apply_only(args, ctx, bt, stream, flush, census, v, w, qv, qtw, world, dev):
    """Q~v + Q~^T w with the transforms already built (as inside a Krylov
    solve), FP32 and FP64, and FP32 with the bead vectors in the tree's
    order, through zq_apply_pair (the two sweeps run concurrently), with the
    sweep bytes achieved against HBM."""
    import torch

    N, R, m = bt.N, bt.n_residues, bt.m
    res = {}
    x, y, z = xyz_of(ctx, bt, dev)
    ctx.pipeline(bt.off, x, y, z, v, qv, w, qtw, level_cut=args.cut)
    ctx.build_transforms(x, y, z)  # both record precisions
    stream.synchronize()
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    for name, dt, es in (("fp32", torch.float32, 4), ("fp64", torch.float64, 8)):
        vv, ww = v.to(dt), w.to(dt)
        oq = torch.empty(R, dtype=dt, device=dev)
        oqt = torch.empty((3, N), dtype=dt, device=dev)
        stream.synchronize()

        def fn():
            ctx.apply_pair(vv, ww, oq, oqt)

        r = timed(args, fn, stream, flush, world, dev, N, graph=not args.no_graph)
        byt = 2 * sweep_bytes(census, N, R, es)
        r["hbm_achieved_gbs"] = byt / (r["ms_per_step"] / 1e3) / 1e9
        r["hbm_frac"] = r["hbm_achieved_gbs"] / hbm
        r["algorithmic_bytes_per_step"] = byt
        res[name] = r
    # bead vectors kept in the tree's sorted-position order (zq_set_vector_order):
    # the sweeps read and write the planes without the gather through perm
    perm = torch.from_numpy(ctx.get_tree()["perm"].astype(np.int64)).to(dev)
    vv, ww = v.to(torch.float32)[:, perm].contiguous(), w.to(torch.float32)
    oq = torch.empty(R, dtype=torch.float32, device=dev)
    oqt = torch.empty((3, N), dtype=torch.float32, device=dev)
    ctx.set_vector_order("tree")
    stream.synchronize()

    def fn_tree():
        ctx.apply_pair(vv, ww, oq, oqt)

    r = timed(args, fn_tree, stream, flush, world, dev, N, graph=not args.no_graph)
    ctx.set_vector_order("caller")
    byt = 2 * sweep_bytes(census, N, R, 4, gather=False)
    r["hbm_achieved_gbs"] = byt / (r["ms_per_step"] / 1e3) / 1e9
    r["hbm_frac"] = r["hbm_achieved_gbs"] / hbm
    r["algorithmic_bytes_per_step"] = byt
    res["fp32_tree_order"] = r
    return res


def qgen_bench(args, ctx, bt, stream, flush, world, dev):
    """The explicit Q~ in CSR form (zq_qgen, Algorithm 1) on the step's batch
    with its transforms built: FP32 and FP64 values.  The bytes counted are
    the CSR written (values, int32 columns, int64 row pointers), the
    kernel's unavoidable traffic; the per-bead path walks read the node
    records through L1/L2."""
    import torch

    N, R = bt.N, bt.n_residues
    x, y, z = xyz_of(ctx, bt, dev)
    ctx.build_tree_batched(bt.off, x, y, z, args.cut)
    ctx.build_transforms(x, y, z)  # both record precisions
    nnz = ctx.qgen_nnz()
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    res = {"nnz": nnz, "nnz_per_bead": nnz / N}
    rp = torch.empty(R + 1, dtype=torch.int64, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    for name, dt, es in (("fp32", torch.float32, 4), ("fp64", torch.float64, 8)):
        val = torch.empty(nnz, dtype=dt, device=dev)

        def fn():
            ctx.qgen_into(rp, col, val)

        r = timed(args, fn, stream, flush, world, dev, N, graph=False, steps=5)
        byt = nnz * (es + 4) + (R + 1) * 8
        r["written_bytes"] = byt
        r["hbm_achieved_gbs"] = byt / (r["ms_per_step"] / 1e3) / 1e9
        r["hbm_frac"] = r["hbm_achieved_gbs"] / hbm
        res[name] = r
        del val
    del rp, col
    torch.cuda.empty_cache()
    return res


def e2e(args, ctx, bt, stream, world, dev):
    """The same step through the C ABI with HOST (pinned) buffers: host to
    device copies of coordinates and vectors, the whole path, and the device
    to host copies of both results inside the timed region."""
    import torch

    N, R = bt.N, bt.n_residues
    rng = np.random.default_rng(7)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hx, hy, hz = pin(bt.x), pin(bt.y), pin(bt.z)
    hv = pin(rng.standard_normal((3, N)).astype(np.float32))
    hw = pin(rng.standard_normal(R).astype(np.float32))
    hq = torch.empty(R, dtype=torch.float32).pin_memory()
    hqt = torch.empty((3, N), dtype=torch.float32).pin_memory()

    def fn():
        ctx.pipeline(bt.off, hx, hy, hz, hv, hq, hw, hqt, level_cut=args.cut, host=True, graph=not args.no_graph)

    for _ in range(2):
        fn()
    ctx.sync()
    steps = max(3, min(args.steps, 10))
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    ms = []
    for _ in range(steps):
        s0.record(stream)
        fn()
        s1.record(stream)
        stream.synchronize()
        ms.append(s0.elapsed_time(s1))
    ctx.sync()
    t = max_over_ranks(world, sum(ms) / 1e3, dev)
    tot = sum_over_ranks(world, float(N) * steps, dev)
    return {"value": tot / t, "unit": "beads/s", "ms_per_step": 1e3 * t / steps,
            "h2d_bytes_per_step": 24 * N + 12 * N + 4 * R, "d2h_bytes_per_step": 4 * R + 12 * N,
            "steps": steps}


# ------------------------------------------------- multi-RHS and BD loop


def multirhs(args, stream, flush, world, dev, rank, k=64):
    """Block form on 500 shells with n_j uniform in [500, 2000] and k = 64
    right-hand sides: Q~V + Q~^T W with the transforms built, in FP32, BF16
    (bfloat16 storage, FP32 arithmetic), FP64, and on the tensor cores (TF32
    and bfloat16 operands, FP32 accumulation, one warp-level mma per node
    and 8-column tile), each with its error against the FP64 oracle on
    sampled columns (rank 0), and FP32 column by column through the
    single-vector path for comparison.  Unit: bead-columns/s."""
    import torch

    import oracle
    from paper_1708_08427_gb300 import workloads as W
    from paper_1708_08427_gb300 import zq

    bt = W.uniform_batch(m=500, nmin=500, nmax=2000, seed=rank)
    N, R = bt.N, bt.n_residues
    x, y, z = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(dev.index, stream)
    ctx.build_tree_batched(bt.off, x, y, z, args.cut)
    ctx.build_transforms(x, y, z)
    census = node_census(ctx)
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    rng = np.random.default_rng(11)
    V64 = torch.from_numpy(rng.standard_normal((3 * N, k))).to(dev)
    W64 = torch.from_numpy(rng.standard_normal((R, k))).to(dev)
    res = {"workload": f"m=500 shells, n_j uniform [500,2000], N={N}, k={k}", "unit": "bead-columns/s"}
    cols = [0, k - 1]
    for name, dt, es, rs, tc in (("fp32", torch.float32, 4, 4, False), ("bf16", torch.bfloat16, 2, 4, False),
                                 ("fp64", torch.float64, 8, 8, False), ("tf32_tensor_core", torch.float32, 4, 4, True),
                                 ("bf16_tensor_core", torch.bfloat16, 2, 4, True)):
        ctx.reserve_block(k, dt)
        V, Wr = V64.to(dt), W64.to(dt)
        oq = torch.empty((R, k), dtype=dt, device=dev)
        oqt = torch.empty((3 * N, k), dtype=dt, device=dev)
        stream.synchronize()

        def fn():
            ctx.apply_Q_block(V, oq, tensor_cores=tc)
            ctx.apply_QT_block(Wr, oqt, tensor_cores=tc)

        r = timed(args, fn, stream, flush, world, dev, N * k, graph=not args.no_graph)
        r["unit"] = "bead-columns/s"
        rec = sum(census[t] * RECORD_FLOATS[t] * rs for t in census)
        nodes = sum(census.values())
        byt = 2 * (k * es * (3 * N + R) + rec + 12 * nodes + 4 * N)
        r["hbm_achieved_gbs"] = byt / (r["ms_per_step"] / 1e3) / 1e9
        r["hbm_frac"] = r["hbm_achieved_gbs"] / hbm
        if rank == 0:
            ctx.sync()
            qv = oq.double().cpu().numpy()
            qtw = oqt.double().cpu().numpy()
            vin = V.double().cpu().numpy()
            win = Wr.double().cpu().numpy()
            err = 0.0
            for c in cols:
                rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z,
                                             W.interleave(*vin[:, c].reshape(3, N)), win[:, c])
                err = max(err, np.linalg.norm(qv[:, c] - rq) / np.linalg.norm(rq),
                          np.linalg.norm(W.interleave(*qtw[:, c].reshape(3, N)) - rqt) / np.linalg.norm(rqt))
            r["rel_err_vs_fp64_oracle"] = err
            r["error_columns"] = cols
        res[name] = r
    # the same work as k single-vector sweeps (FP32), for comparison
    Vc = V64.t().contiguous().to(torch.float32).reshape(k, 3, N)
    Wc = W64.t().contiguous().to(torch.float32)
    oqc = torch.empty((k, R), dtype=torch.float32, device=dev)
    oqtc = torch.empty((k, 3, N), dtype=torch.float32, device=dev)

    def fn_cols():
        ctx.apply_Q(Vc, oqc)
        ctx.apply_QT(Wc, oqtc)

    r = timed(args, fn_cols, stream, flush, world, dev, N * k, graph=not args.no_graph, steps=3)
    r["unit"] = "bead-columns/s"
    res["fp32_column_by_column"] = r
    ctx.close()
    return res


def ellipsoid_leg(args, stream, flush, world, dev, rank):
    """One body of 2^20 beads (the ellipsoid with semi-axes (3, 2, 1) sqrt(n)/100
    and radial jitter N(0, 0.01^2)): the same step (tree, double-single
    transforms, FP32 Q~v and Q~^T w, one zq_pipeline call replayed from the
    library's graph), each level cut of the tuner timed; the body is too
    large for the fused step.  Its per-bead rate against the batched step
    shows the cost of the large-body path."""
    import torch

    from paper_1708_08427_gb300 import workloads as W
    from paper_1708_08427_gb300 import zq
    from paper_1708_08427_gb300.tune import tune_level_cut

    bt = W.ellipsoid_body(n=1 << 20, seed=rank)
    N, R = bt.N, bt.n_residues
    rng = np.random.default_rng(5)
    with torch.cuda.stream(stream):
        x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
        v = torch.from_numpy(rng.standard_normal((3, N))).to(dev, torch.float32)
        w = torch.from_numpy(rng.standard_normal(R)).to(dev, torch.float32)
        qv = torch.empty(R, device=dev)
        qtw = torch.empty((3, N), device=dev)
    stream.synchronize()
    ctx = zq.Context(dev.index, stream)
    cut, times = tune_level_cut(ctx, bt.off, x, y, z, v, qv, w, qtw, graph=not args.no_graph)

    def fn():
        ctx.pipeline(bt.off, x, y, z, v, qv, w, qtw, level_cut=cut, graph=not args.no_graph)

    r = timed(args, fn, stream, flush, world, dev, N, graph=False)
    ctx.close()
    r.update({"workload": "one ellipsoid body, n=2^20, semi-axes (3,2,1)*sqrt(n)/100, radial jitter N(0,0.01^2)",
              "level_cut": cut, "level_cut_tuning_ms": times})
    return r


def bd_loop(args, stream, flush, world, dev, rank, steps_in_graph=10, reuse=False):
    """Brownian-dynamics style loop on 1000 shells of 1000 beads with the tree
    kept: per step every body gets a rigid motion (unit quaternion from
    normalised N(0, I_4) about its centroid, N(0, 0.1^2) translation; applied
    with torch as the workload driver) and Q~^T (Q~ f) is computed in FP32
    for an N(0, 1) force f.  reuse=False: the transforms are rebuilt on the
    kept tree every step.  reuse=True: the transforms of the first positions
    are kept and every body's accumulated rotation is applied to the bead
    vectors instead (zq_apply_rotated).  The loop is captured in a CUDA
    graph (steps_in_graph steps per replay).  The projector error
    |Q~^T Q~ f - (f - Z^T (Z Z^T)^-1 Z f)| / |f| is measured (FP64, torch)
    after the timed replays."""
    import torch

    from paper_1708_08427_gb300 import workloads as W
    from paper_1708_08427_gb300 import zq

    m, n = 1000, 1000
    bt = W.fixed_batch(m=m, n=n, seed=rank)
    N, R = bt.N, bt.n_residues
    body = torch.arange(m, device=dev).repeat_interleave(n)
    P = torch.from_numpy(np.stack([bt.x, bt.y, bt.z], 1)).to(dev)          # (N, 3) float64
    ctx = zq.Context(dev.index, stream)
    x, y, z = (P[:, a].contiguous() for a in range(3))
    ctx.build_tree_batched(bt.off, x, y, z, args.cut)
    ctx.build_transforms(x, y, z)
    torch.cuda.manual_seed(1234 + rank)  # the default generator: CUDA-graph safe
    f = torch.empty((3, N), dtype=torch.float32, device=dev)
    qf = torch.empty(R, dtype=torch.float32, device=dev)
    out = torch.empty((3, N), dtype=torch.float32, device=dev)

    def rot(q):  # (m, 4) unit quaternions -> (m, 3, 3)
        a, b, c, d = q.unbind(1)
        return torch.stack([
            torch.stack([a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)], 1),
            torch.stack([2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)], 1),
            torch.stack([2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d], 1)], 1)

    Racc = torch.eye(3, dtype=torch.float64, device=dev).repeat(m, 1, 1).contiguous()

    def one_step():
        q = torch.randn((m, 4), device=dev, dtype=torch.float64)
        q = q / q.norm(dim=1, keepdim=True)
        t = 0.1 * torch.randn((m, 3), device=dev, dtype=torch.float64)
        P3 = P.view(m, n, 3)
        cen = P3.mean(1, keepdim=True)
        Rq = rot(q)
        P3.copy_(torch.bmm(P3 - cen, Rq.transpose(1, 2)) + cen + t[:, None, :])
        f.copy_(torch.randn((3, N), device=dev, dtype=torch.float32))
        if reuse:
            Racc.copy_(torch.bmm(Rq, Racc))
            ctx.apply_rotated(Racc, v=f, qv=qf)
            ctx.apply_rotated(Racc, w=qf, qtw=out)
        else:
            x.copy_(P[:, 0]); y.copy_(P[:, 1]); z.copy_(P[:, 2])
            ctx.build_transforms(x, y, z)
            ctx.apply_Q(f, qf)
            ctx.apply_QT(qf, out)

    for _ in range(2):
        with torch.cuda.stream(stream):
            one_step()
    stream.synchronize()
    g = None
    if not args.no_graph:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(steps_in_graph):
                one_step()
        stream.synchronize()
    def run_replay():
        with torch.cuda.stream(stream):
            if g is not None:
                g.replay()
            else:
                for _ in range(steps_in_graph):
                    one_step()

    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20  # 200 steps
    s0.record(stream)
    for _ in range(reps):
        run_replay()
    s1.record(stream)
    stream.synchronize()
    ctx.sync()
    t_step = max_over_ranks(world, s0.elapsed_time(s1) / 1e3, dev) / (reps * steps_in_graph)

    def projector_err():
        """|Q~^T Q~ f - (f - Z^T (Z Z^T)^-1 Z f)| / |f| of the last step, FP64."""
        Pc = P - (torch.zeros((m, 3), device=dev, dtype=torch.float64).index_add_(0, body, P) / n)[body]
        fd = f.double().t()                                            # (N, 3)
        Fsum = torch.zeros((m, 3), device=dev, dtype=torch.float64).index_add_(0, body, fd)
        Tsum = torch.zeros((m, 3), device=dev, dtype=torch.float64).index_add_(0, body, torch.cross(Pc, fd, dim=1))
        r2 = (Pc * Pc).sum(1)
        J = torch.zeros((m, 3, 3), device=dev, dtype=torch.float64).index_add_(
            0, body, r2[:, None, None] * torch.eye(3, device=dev, dtype=torch.float64)
            - Pc[:, :, None] * Pc[:, None, :])
        om = torch.linalg.solve(J, Tsum)
        Pf = (Fsum / n)[body] + torch.cross(om[body], Pc, dim=1)
        return float(((out.double().t() - (fd - Pf)).norm() / fd.norm()).item())

    def oracle_spot(bodies):
        """The same projector from the FP64 oracle's own tree and transforms
        on the moved positions (Q~^T Q~ does not depend on the basis), for a
        few bodies: worst relative error of the GPU's FP32 result."""
        import oracle
        from paper_1708_08427_gb300 import workloads as W

        Ph = P.cpu().numpy()
        fh = f.double().cpu().numpy()
        oh = out.double().cpu().numpy()
        worst = 0.0
        for j in bodies:
            a, b = j * n, (j + 1) * n
            B = oracle.Body(Ph[a:b, 0].copy(), Ph[a:b, 1].copy(), Ph[a:b, 2].copy())
            fj = W.interleave(*fh[:, a:b])
            want = B.apply_QT(B.apply_Q(fj))
            got = W.interleave(*oh[:, a:b])
            worst = max(worst, float(np.linalg.norm(got - want) / np.linalg.norm(fj)))
        return worst

    # sampled steps after the timed ones: the last step of each of three
    # more replays, checked in full (FP64 torch) and by the oracle on 8 bodies
    errs, spots = [], []
    rs = np.random.default_rng(77)
    for _ in range(3):
        run_replay()
        stream.synchronize()
        errs.append(projector_err())
        if rank == 0:
            spots.append(oracle_spot(sorted(rs.choice(m, 8, replace=False).tolist())))
    ctx.close()
    what = ("transforms kept, accumulated rotation applied to the bead vectors" if reuse
            else "transforms rebuilt")
    return {"workload": f"m=1000 shells x 1000 beads, tree kept, per step: rigid motion, {what}, "
                        "Q~^T(Q~ f) FP32", "steps_per_s": 1.0 / t_step, "ms_per_step": 1e3 * t_step,
            "beads_per_s": N / t_step, "graph": g is not None, "steps_timed": reps * steps_in_graph,
            "projector_rel_err_fp32": max(errs), "projector_rel_err_sampled_steps": errs,
            "oracle_spot_check_rel_err": spots,
            "oracle_spot_check": "8 bodies per sampled step, the oracle's own Q~^T Q~ f on the moved positions"}


# ------------------------------------------------------------ CPU oracle


def oracle_sample(bt, seconds: float):
    """A prefix of the batch sized to about `seconds` of oracle work."""
    import oracle

    probe = max(1, min(bt.m, 20))
    t0 = time.perf_counter()
    n_probe = int(bt.off[probe])
    _oracle_step(bt, probe, np.random.default_rng(0))
    dt = time.perf_counter() - t0
    rate = n_probe / max(dt, 1e-6)
    target = rate * seconds
    nb = int(np.searchsorted(bt.off, target))
    return max(1, min(bt.m, nb)), rate


def _oracle_step(bt, nbodies, rng):
    import oracle

    off = bt.off[:nbodies + 1]
    n = int(off[-1])
    f = rng.standard_normal(3 * n)
    w = rng.standard_normal(3 * n - 6 * nbodies)
    oracle.batch_apply(off, bt.x[:n], bt.y[:n], bt.z[:n], f, w)
    return n


def cpu_baseline(bt, seconds):
    nb, _ = oracle_sample(bt, seconds)
    rng = np.random.default_rng(1)
    t0 = time.perf_counter()
    n = _oracle_step(bt, nb, rng)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "beads/s", "cores": 1, "kind": "oracle",
            "sample": f"first {nb} of {bt.m} bodies ({n} beads): tree + FP64 transforms + Q~v + "
                      f"Q~^T w, single-threaded C, {dt:.1f} s", "host_cpus": os.cpu_count()}


def run_reference(args, world, rank):
    """The oracle as the reference arm: the same metric on host cores, each
    step a bounded sample of the workload."""
    if rank != 0:
        return None
    bt, desc = make_workload(args.workload, seed=0, bodies=args.bodies)
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    nb, _ = oracle_sample(bt, per_step)
    rng = np.random.default_rng(3)
    for _ in range(args.warmup):
        _oracle_step(bt, nb, rng)
    t0 = time.perf_counter()
    n_tot = 0
    for _ in range(args.steps):
        n_tot += _oracle_step(bt, nb, rng)
    dt = time.perf_counter() - t0
    val = n_tot / dt
    return {"metric": METRIC, "value": val, "unit": "beads/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded numpy generators; no dataset)",
            "config": {"workload": desc, "m": bt.m, "N": bt.N, "sample_bodies": nb},
            "cpu_baseline": {"value": val, "unit": "beads/s", "kind": "oracle", "cores": 1,
                             "sample": f"first {nb} of {bt.m} bodies per step, single-threaded C"},
            "e2e": {"value": val, "unit": "beads/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        out = run_reference(args, world, rank)
    else:
        out = run_ours(args, world, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
