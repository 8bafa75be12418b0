"""Body sharding over two CPU ranks (gloo): each rank applies Q~ to its
own bodies (the FP64 oracle stands in for the GPU sweeps, which need a
device); the gathered slices equal the single-process result exactly, the
shards cover every body once, and LPT keeps each rank within one largest
body of the average load."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import oracle
    from paper_1708_08427_gb300 import shard
    from paper_1708_08427_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bt = W.shell_batch(m=23, nmin=20, nmax=400, seed=4)
    sub, bodies = shard.shard(bt, world, rank)
    rng = np.random.default_rng(9)
    f = rng.standard_normal(3 * bt.N)
    w = rng.standard_normal(bt.n_residues)
    # this rank's slices of the global inputs
    fl = np.concatenate([f[3 * b0:3 * b1] for (b0, b1), _ in shard.global_slices(bt, bodies)])
    wl = np.concatenate([w[r0:r1] for _, (r0, r1) in shard.global_slices(bt, bodies)])
    qv, qtw = oracle.batch_apply(sub.off, sub.x, sub.y, sub.z, fl, wl)
    parts = [None] * world
    dist.all_gather_object(parts, (bodies, qv, qtw))
    if rank == 0:
        gq = np.full(bt.n_residues, np.nan)
        gqt = np.full(3 * bt.N, np.nan)
        for b, lq, lqt in parts:
            shard.place(bt, b, lq, gq)
            pos = 0
            for (b0, b1), _ in shard.global_slices(bt, b):
                gqt[3 * b0:3 * b1] = lqt[pos:pos + 3 * (b1 - b0)]
                pos += 3 * (b1 - b0)
        rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, f, w)
        allb = np.sort(np.concatenate([p[0] for p in parts]))
        loads = [int(bt.sizes[p[0]].sum()) for p in parts]
        q.put((np.array_equal(allb, np.arange(bt.m)), bool(np.array_equal(gq, rq)),
               bool(np.array_equal(gqt, rqt)), loads, int(bt.sizes.max()), int(bt.N)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_matches_single_process():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        cover, eq_q, eq_qt, loads, biggest, N = q.get(timeout=240)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert cover and eq_q and eq_qt
    assert max(loads) <= N / world + biggest


def test_lpt_partition_properties():
    from paper_1708_08427_gb300 import shard

    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        sizes = rng.integers(3, 5000, size=97)
        parts = shard.lpt_partition(sizes, world)
        assert sorted(np.concatenate(parts).tolist()) == list(range(97))
        loads = [int(sizes[p].sum()) for p in parts]
        assert max(loads) <= sizes.sum() / world + sizes.max()
