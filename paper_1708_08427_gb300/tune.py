"""Autotuning of the step's schedule: the level schedule at each candidate
level cut (heights 1..cut as one launch per height over all bodies, the
heights above one block or warp per body; sweeps on 512-bead segments), or
the fused per-body step (one persistent launch, one thread block per body;
bodies of at most 8192 beads).  Results do not depend on the choice (the
same bits); only the time does.

The tuner times the whole step (zq_pipeline: tree, transforms, both sweeps)
on the caller's workload for each candidate with CUDA events on the
context's stream and returns the fastest, with the times it measured.
Picks can be kept in a JSON cache keyed by the workload's shape (body-size
histogram in powers of two, total beads, precision, build arithmetic,
vector order, graph replay), so a later run on the same shape skips the
timing.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

import numpy as np

CUTS = (9, 12, 15, 18, 21)
# candidates: ("levels", cut) for every cut, and ("fused", 0)
CANDIDATES = tuple(("levels", c) for c in CUTS) + (("fused", 0),)


def shape_key(off, prec: str, arith: str, order: str, graph: bool) -> str:
    """A key for the workload's shape: body sizes binned by powers of two."""
    n = np.diff(np.asarray(off, dtype=np.int64))
    hist = np.bincount(np.floor(np.log2(n)).astype(np.int64), minlength=1)
    return json.dumps({"m": int(n.size), "N": int(n.sum()), "log2_hist": hist.tolist(), "prec": prec,
                       "arith": arith, "order": order, "graph": bool(graph)}, sort_keys=True)


def _load(cache: Path | None) -> dict:
    if cache is None or not cache.exists():
        return {}
    try:
        return json.loads(cache.read_text())
    except (OSError, ValueError):
        return {}


def tune_step(ctx, off, x, y, z, v, qv, w, qtw, candidates=CANDIDATES, reps: int = 5, warmup: int = 2,
              graph: bool = False, cache: str | os.PathLike | None = None, key_extra: dict | None = None):
    """Returns ((schedule, cut), {"schedule:cut": ms per step}, from_cache).
    graph: time the step as the library's CUDA-graph replay (ZQ_GRAPH), the
    way it will then run.  cache: a JSON file of earlier picks (read, and
    written with this pick)."""
    import torch

    path = Path(cache) if cache else None
    prec = "fp64" if qv is not None and qv.dtype == torch.float64 else "fp32"
    extra = key_extra or {}
    key = shape_key(off, prec, extra.get("arith", "dd"), extra.get("order", "caller"), graph)
    known = _load(path)
    if key in known:
        s, c = known[key]["pick"]
        ctx.set_step_schedule(s)
        return (s, int(c)), known[key]["times"], True
    stream = ctx.stream
    times = {}
    for sched, cut in candidates:
        ctx.set_step_schedule(sched)
        for _ in range(warmup):  # with graph: plan, then capture
            ctx.pipeline(off, x, y, z, v, qv, w, qtw, level_cut=cut, graph=graph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.pipeline(off, x, y, z, v, qv, w, qtw, level_cut=cut, graph=graph)
        e1.record(stream)
        e1.synchronize()
        ctx.sync()
        times[f"{sched}:{cut}"] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    s, c = best.split(":")
    ctx.set_step_schedule(s)
    if path is not None:
        known[key] = {"pick": [s, int(c)], "times": times}
        path.parent.mkdir(parents=True, exist_ok=True)
        tmp = path.with_suffix(f".{os.getpid()}.tmp")
        tmp.write_text(json.dumps(known, indent=1, sort_keys=True))
        os.replace(tmp, path)
    return (s, int(c)), times, False


def tune_level_cut(ctx, off, x, y, z, v, qv, w, qtw, cuts=CUTS, reps: int = 5, warmup: int = 2,
                   graph: bool = False):
    """The level schedule only: returns (best cut, {cut: ms per step})."""
    (_, best), times, _ = tune_step(ctx, off, x, y, z, v, qv, w, qtw, candidates=tuple(("levels", c) for c in cuts),
                                    reps=reps, warmup=warmup, graph=graph)
    return best, {int(k.split(":")[1]): t for k, t in times.items()}
