"""Autotuning of the level cut (the one schedule knob of the node-transform
build: heights 1..cut run as one launch per height over all bodies, the
heights above one thread block per body).  Results do not depend on the
cut; only the time does.

The tuner times the whole step (zq_pipeline: tree, transforms, both sweeps)
on the caller's workload for each candidate cut with CUDA events on the
context's stream and returns the fastest, with the times it measured.
"""
from __future__ import annotations

CUTS = (9, 12, 15, 18, 21)


def tune_level_cut(ctx, off, x, y, z, v, qv, w, qtw, cuts=CUTS, reps: int = 5, warmup: int = 2,
                   graph: bool = False):
    """Returns (best cut, {cut: ms per step}).  graph: time the step as the
    library's CUDA-graph replay (ZQ_GRAPH), the way it will then run."""
    import torch

    stream = ctx.stream
    times = {}
    for cut in cuts:
        for _ in range(warmup):  # with graph: plan, then capture
            ctx.pipeline(off, x, y, z, v, qv, w, qtw, level_cut=cut, graph=graph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.pipeline(off, x, y, z, v, qv, w, qtw, level_cut=cut, graph=graph)
        e1.record(stream)
        e1.synchronize()
        ctx.sync()
        times[cut] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    return best, times
