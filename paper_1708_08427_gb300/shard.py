"""Sharding a batch of bodies over ranks (one process per GPU).

Q~ of a batch is block diagonal, one block per body (Sec. 1), so Q~v and
Q~^T w of different bodies never interact: a batch splits over ranks body by
body with no exchange in the data path.  Bodies go to ranks by longest
processing time first (the largest remaining body to the least loaded rank,
load = beads), which keeps every rank within one largest body of the
average.  Each rank builds the tree and transforms of its own bodies and
writes its slice of the global result; the slices are disjoint and their
offsets follow from the body sizes alone.

Host logic only (numpy); no GPU, no collective.
"""
from __future__ import annotations

import heapq

import numpy as np

from .workloads import Batch


def lpt_partition(sizes: np.ndarray, world: int) -> list[np.ndarray]:
    """Body indices of each rank (ascending), by longest processing time
    first on the bead counts."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for j in np.argsort(-sizes, kind="stable"):
        load, r = heapq.heappop(heap)
        parts[r].append(int(j))
        heapq.heappush(heap, (load + int(sizes[j]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def sub_batch(bt: Batch, bodies: np.ndarray) -> Batch:
    """The bodies (global indices, ascending) as a batch of their own."""
    sizes = bt.sizes[bodies]
    off = np.zeros(len(bodies) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    idx = np.concatenate([np.arange(bt.off[j], bt.off[j + 1]) for j in bodies]) if len(bodies) else \
        np.zeros(0, np.int64)
    return Batch(off, bt.x[idx].copy(), bt.y[idx].copy(), bt.z[idx].copy())


def shard(bt: Batch, world: int, rank: int) -> tuple[Batch, np.ndarray]:
    """This rank's bodies (global indices) and their batch."""
    bodies = lpt_partition(bt.sizes, world)[rank]
    return sub_batch(bt, bodies), bodies


def global_slices(bt: Batch, bodies: np.ndarray):
    """For each of the given bodies: (bead range, residue range) in the
    global vectors (beads [off_j, off_{j+1}); residues of body j start at
    sum_{i<j} (3 n_i - 6))."""
    roff = np.zeros(bt.m + 1, np.int64)
    roff[1:] = np.cumsum(3 * bt.sizes - 6)
    return [((int(bt.off[j]), int(bt.off[j + 1])), (int(roff[j]), int(roff[j + 1]))) for j in bodies]


def place(bt: Batch, bodies: np.ndarray, local_res: np.ndarray, global_res: np.ndarray) -> None:
    """Copy a rank's residue vector (its bodies in ascending order) into the
    global residue vector."""
    pos = 0
    for _, (r0, r1) in global_slices(bt, bodies):
        global_res[r0:r1] = local_res[pos:pos + (r1 - r0)]
        pos += r1 - r0
