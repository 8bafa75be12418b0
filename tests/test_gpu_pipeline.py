"""zq_pipeline, the one-call step the benchmark times: tree, transforms and
both products (Q~v on the context stream, Q~^T w concurrently on a side
stream with its own scratch), from device or pinned host buffers, with the
tree rebuilt or kept.

Against the FP64 oracle per body (1e-12 FP64, 1e-5 FP32), by each body's
relative 2-norm and element by element.  With the tree
kept, the oracle's own tree (built from the moved coordinates) is not the
kept one, so the result is checked against the separate calls on a context
that built its tree from the original coordinates (bitwise), and against
the basis-free projector identity Q~^T Q~ f = f - Z^T (Z Z^T)^-1 Z f.
"""
import numpy as np
import pytest

import oracle
from _parity import compare_per_body
from paper_1708_08427_gb300 import tune
from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _zq():
    from paper_1708_08427_gb300 import zq

    return zq


@pytest.mark.parametrize("dtype,host", [(torch.float32, False), (torch.float64, False), (torch.float32, True)])
def test_pipeline_matches_oracle(dtype, host):
    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=24, nmin=20, nmax=1800, seed=31)
    rng = np.random.default_rng(2)
    v = rng.standard_normal((3, bt.N))
    w = rng.standard_normal(bt.n_residues)
    if host:
        mk = lambda a, dt=dtype: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
        x, y, z = (mk(a, torch.float64) for a in (bt.x, bt.y, bt.z))
        tv, tw = mk(v), mk(w)
        qv = torch.empty(bt.n_residues, dtype=dtype).pin_memory()
        qtw = torch.empty((3, bt.N), dtype=dtype).pin_memory()
    else:
        mk = lambda a, dt=dtype: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
        x, y, z = (mk(a, torch.float64) for a in (bt.x, bt.y, bt.z))
        tv, tw = mk(v), mk(w)
        qv = torch.empty(bt.n_residues, dtype=dtype, device=dev)
        qtw = torch.empty((3, bt.N), dtype=dtype, device=dev)
    ctx = zq.Context(0)
    for _ in range(2):  # a second call reuses the plan and the buffers
        ctx.pipeline(bt.off, x, y, z, tv, qv, tw, qtw, host=host)
        ctx.sync()
        rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, W.interleave(*v), w)
        compare_per_body(qv.double().cpu().numpy(), rq, bt.off, "res", TOL[dtype], "Q~v")
        compare_per_body(W.interleave(*qtw.double().cpu().numpy()), rqt, bt.off, "bead", TOL[dtype], "Q~^T w")
    ctx.close()


def test_pipeline_single_products_match_pair():
    """Only Q~v, only Q~^T w, and both at once give the same bits."""
    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=9, nmin=30, nmax=900, seed=5)
    rng = np.random.default_rng(8)
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    v = torch.from_numpy(rng.standard_normal((3, bt.N))).to(dev, torch.float32)
    w = torch.from_numpy(rng.standard_normal(bt.n_residues)).to(dev, torch.float32)
    out = {}
    for mode in ("both", "v", "w"):
        ctx = zq.Context(0)
        qv = torch.full((bt.n_residues,), float("nan"), device=dev)
        qtw = torch.full((3, bt.N), float("nan"), device=dev)
        ctx.pipeline(bt.off, x, y, z, v if mode != "w" else None, qv if mode != "w" else None,
                     w if mode != "v" else None, qtw if mode != "v" else None)
        ctx.sync()
        out[mode] = (qv.cpu(), qtw.cpu())
        ctx.close()
    assert torch.equal(out["both"][0], out["v"][0])
    assert torch.equal(out["both"][1], out["w"][1])


def _projector_residual(P, f, off):
    """|f - Z^T (Z Z^T)^-1 Z f| per body, P (N, 3) positions, f (N, 3)."""
    res = np.empty_like(f)
    for j in range(len(off) - 1):
        a, b = off[j], off[j + 1]
        p = P[a:b] - P[a:b].mean(0)
        g = f[a:b]
        J = (p * p).sum() * np.eye(3) - p.T @ p
        om = np.linalg.solve(J, np.cross(p, g).sum(0))
        res[a:b] = g - (g.mean(0) + np.cross(om, p))
    return res


def test_pipeline_keep_tree_after_rigid_motion():
    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=12, nmin=40, nmax=1200, seed=13)
    qs, ts = W.random_rigid_motions(bt.m, 1, seed=4)
    P = np.stack([bt.x, bt.y, bt.z], 1)
    Pm = P.copy()
    for j in range(bt.m):
        a, b = bt.off[j], bt.off[j + 1]
        q0, q1, q2, q3 = qs[0, j]
        R = np.array([[q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, 2 * (q1 * q2 - q0 * q3), 2 * (q1 * q3 + q0 * q2)],
                      [2 * (q1 * q2 + q0 * q3), q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3, 2 * (q2 * q3 - q0 * q1)],
                      [2 * (q1 * q3 - q0 * q2), 2 * (q2 * q3 + q0 * q1), q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3]])
        c = P[a:b].mean(0)
        Pm[a:b] = (P[a:b] - c) @ R.T + c + ts[0, j]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x0, y0, z0 = d(P[:, 0]), d(P[:, 1]), d(P[:, 2])
    x1, y1, z1 = d(Pm[:, 0]), d(Pm[:, 1]), d(Pm[:, 2])
    rng = np.random.default_rng(3)
    f = rng.standard_normal((3, bt.N))
    v = d(f)
    ctx = zq.Context(0)
    qv = torch.empty(bt.n_residues, dtype=torch.float64, device=dev)
    out = torch.empty((3, bt.N), dtype=torch.float64, device=dev)
    ctx.pipeline(bt.off, x0, y0, z0, v, qv)                      # tree from the original positions
    ctx.pipeline(bt.off, x1, y1, z1, v, qv, keep_tree=True)      # moved beads, kept tree
    ctx.apply_QT(qv, out)
    ctx.sync()
    ref = zq.Context(0)
    ref.build_tree_batched(bt.off, x0, y0, z0)
    ref.build_transforms(x1, y1, z1)
    rqv = ref.apply_Q(v)
    ref.sync()
    assert torch.equal(qv, rqv)
    got = out.cpu().numpy().T
    want = _projector_residual(Pm, f.T, bt.off)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(f).max() * 10
    ctx.close()
    ref.close()


def test_apply_pair_equals_separate_calls():
    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=10, nmin=30, nmax=1500, seed=17)
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    rng = np.random.default_rng(21)
    ctx = zq.Context(0)
    ctx.build_tree_batched(bt.off, x, y, z)
    ctx.build_transforms(x, y, z)
    for dt in (torch.float32, torch.float64):
        v = torch.from_numpy(rng.standard_normal((3, bt.N))).to(dev, dt)
        w = torch.from_numpy(rng.standard_normal(bt.n_residues)).to(dev, dt)
        qv, qtw = ctx.apply_pair(v, w)
        rqv, rqtw = ctx.apply_Q(v), ctx.apply_QT(w)
        ctx.sync()
        assert torch.equal(qv, rqv) and torch.equal(qtw, rqtw)
    ctx.close()


def test_level_cut_tuner_picks_a_candidate():
    from paper_1708_08427_gb300.tune import tune_level_cut

    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=16, nmin=30, nmax=2000, seed=23)
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    v = torch.zeros((3, bt.N), device=dev)
    w = torch.zeros(bt.n_residues, device=dev)
    qv = torch.empty(bt.n_residues, device=dev)
    qtw = torch.empty((3, bt.N), device=dev)
    ctx = zq.Context(0)
    best, times = tune_level_cut(ctx, bt.off, x, y, z, v, qv, w, qtw, cuts=(4, 15), reps=2, warmup=1)
    assert best in (4, 15) and set(times) == {4, 15} and all(t > 0 for t in times.values())
    ctx.close()


def test_step_tuner_picks_a_candidate_and_caches_it(tmp_path):
    """tune_step times the level schedule at two cuts and the fused step,
    leaves the context on the fastest schedule, writes the pick to the cache
    and takes it from there on the next call."""
    from paper_1708_08427_gb300.tune import tune_step

    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=16, nmin=30, nmax=2000, seed=23)
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    v = torch.zeros((3, bt.N), device=dev)
    w = torch.zeros(bt.n_residues, device=dev)
    qv = torch.empty(bt.n_residues, device=dev)
    qtw = torch.empty((3, bt.N), device=dev)
    ctx = zq.Context(0)
    cands = (("levels", 4), ("levels", 15), ("fused", 0))
    cache = tmp_path / "picks.json"
    pick, times, cached = tune_step(ctx, bt.off, x, y, z, v, qv, w, qtw, candidates=cands, reps=2, warmup=1,
                                    cache=cache)
    assert not cached and pick in [(s, c) for s, c in cands] and len(times) == 3
    assert cache.exists()
    pick2, times2, cached2 = tune_step(ctx, bt.off, x, y, z, v, qv, w, qtw, candidates=cands, cache=cache)
    assert cached2 and pick2 == pick and times2 == times
    ctx.close()


@pytest.mark.parametrize("host", [False, True])
def test_pipeline_graph_replay_matches_direct(host):
    """ZQ_GRAPH: the first call plans and runs directly, the second captures,
    later calls replay; every call gives the bits of the direct path, also
    after the inputs change in place.  A call with other arguments or after
    a new plan is not replayed from the stale graph."""
    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=16, nmin=20, nmax=2500, seed=41)
    rng = np.random.default_rng(43)
    if host:
        mk = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
        out = lambda shape: torch.empty(shape, dtype=torch.float32).pin_memory()
    else:
        mk = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
        out = lambda shape: torch.empty(shape, dtype=torch.float32, device=dev)
    x, y, z = (mk(a, torch.float64) for a in (bt.x, bt.y, bt.z))
    v, w = mk(rng.standard_normal((3, bt.N))), mk(rng.standard_normal(bt.n_residues))
    qv, qtw = out(bt.n_residues), out((3, bt.N))
    g = zq.Context(0, torch.cuda.Stream(dev))  # a capturable (non-default) stream
    d = zq.Context(0, torch.cuda.Stream(dev))
    torch.cuda.synchronize()
    l0 = None
    for it in range(4):
        if it == 2:  # new inputs in place: the replay reads them
            v.copy_(mk(rng.standard_normal((3, bt.N))))
            x.copy_(mk(bt.x + 0.01 * rng.standard_normal(bt.N), torch.float64))
            torch.cuda.synchronize()
        g.pipeline(bt.off, x, y, z, v, qv, w, qtw, host=host, graph=True)
        g.sync()
        rq, rqt = out(bt.n_residues), out((3, bt.N))
        d.pipeline(bt.off, x, y, z, v, rq, w, rqt, host=host)
        d.sync()
        assert torch.equal(qv, rq) and torch.equal(qtw, rqt), it
        n = g.launch_count()
        if l0 is not None and it >= 2:
            assert n - l0 > 0  # a replay counts the step's kernels
        l0 = n
    # another batch on the same context: planned afresh, not the old graph
    bt2 = W.shell_batch(m=7, nmin=20, nmax=900, seed=44)
    x2, y2, z2 = (mk(a, torch.float64) for a in (bt2.x, bt2.y, bt2.z))
    v2 = mk(rng.standard_normal((3, bt2.N)))
    q2, r2 = out(bt2.n_residues), out(bt2.n_residues)
    torch.cuda.synchronize()
    for _ in range(3):
        g.pipeline(bt2.off, x2, y2, z2, v2, q2, host=host, graph=True)
        g.sync()
    d.pipeline(bt2.off, x2, y2, z2, v2, r2, host=host)
    d.sync()
    assert torch.equal(q2, r2)
    g.close()
    d.close()


@pytest.mark.parametrize("cut", tune.CUTS)
def test_full_size_step_as_benched(cut):
    """The benchmark's step exactly as bench.py times it: the 2000-shell
    batch (2,155,957 beads, seed 0), one zq_pipeline call per step in FP32
    with the double-single build, on a non-default stream, replayed from the
    library's CUDA graph (ZQ_GRAPH), at every level cut the tuner can pick.
    The third call is a replay; every output of it is checked per body
    against the FP64 oracle (1e-5), by norm and element by element."""
    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=2000, nmin=50, nmax=5000, seed=0)
    rng = np.random.default_rng(1000)
    v = rng.standard_normal((3, bt.N))
    w = rng.standard_normal(bt.n_residues)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
        tv = torch.from_numpy(v).to(dev, torch.float32)
        tw = torch.from_numpy(w).to(dev, torch.float32)
        qv = torch.empty(bt.n_residues, device=dev)
        qtw = torch.empty((3, bt.N), device=dev)
    stream.synchronize()
    ctx = zq.Context(0, stream=stream)
    ctx.set_build_arith("dd")
    for _ in range(3):  # plan, capture, replay
        with torch.cuda.stream(stream):  # ordered before the call on its stream
            qv.fill_(float("nan"))
            qtw.fill_(float("nan"))
        ctx.pipeline(bt.off, x, y, z, tv, qv, tw, qtw, level_cut=cut, graph=True)
    ctx.sync()
    # the oracle sees the FP32-rounded inputs the kernels saw
    vr = tv.double().cpu().numpy()
    wr = tw.double().cpu().numpy()
    rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, W.interleave(*vr), wr)
    compare_per_body(qv.double().cpu().numpy(), rq, bt.off, "res", TOL[torch.float32], f"Q~v cut {cut}")
    compare_per_body(W.interleave(*qtw.double().cpu().numpy()), rqt, bt.off, "bead", TOL[torch.float32],
                     f"Q~^T w cut {cut}")
    ctx.close()
