"""The fused step of zq_pipeline (zq_set_step_schedule(ZQ_STEP_FUSED)): the
transforms, Q~v and Q~^T w of every body in one persistent launch, one
thread block per body (bodies are independent: Q~ is block diagonal, Sec. 1).

The node arithmetic is the level schedule's, so both schedules must give
the same bits, in every precision, build arithmetic and vector order, with
one product or both, from device or host buffers and replayed from a
graph.  The benched configuration (2000 shells, FP32 products,
double-single build, graph replay) is also checked against the FP64
oracle by norm and element by element.  After a fused step the separate
products need zq_build_transforms; a batch with a body over 8192 beads
falls back to the level schedule.
"""
import numpy as np
import pytest

import oracle
from _parity import compare_per_body
from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _zq():
    from paper_1708_08427_gb300 import zq

    return zq


def _run(bt, schedule, dtype, arith="dd", order="caller", graph=False, products="both", host=False, reps=1,
         seed=3):
    zq = _zq()
    dev = _dev()
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3, bt.N))
    w = rng.standard_normal(bt.n_residues)
    if host:
        mk = lambda a, dt=dtype: torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
        out = lambda shape: torch.full(shape, float("nan"), dtype=dtype).pin_memory()
    else:
        mk = lambda a, dt=dtype: torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)
        out = lambda shape: torch.full(shape, float("nan"), dtype=dtype, device=dev)
    x, y, z = (mk(a, torch.float64) for a in (bt.x, bt.y, bt.z))
    tv, tw = mk(v), mk(w)
    qv, qtw = out((bt.n_residues,)), out((3, bt.N))
    ctx = zq.Context(0, torch.cuda.Stream(dev))
    ctx.set_build_arith(arith)
    ctx.set_step_schedule(schedule)
    ctx.set_vector_order(order)
    torch.cuda.synchronize()
    for _ in range(reps):
        ctx.pipeline(bt.off, x, y, z, tv if products != "w" else None, qv if products != "w" else None,
                     tw if products != "v" else None, qtw if products != "v" else None, host=host, graph=graph)
    ctx.sync()
    res = (qv.cpu().clone(), qtw.cpu().clone())
    ctx.close()
    return res, v, w


@pytest.mark.parametrize("dtype,arith", [(torch.float32, "dd"), (torch.float64, "dd"), (torch.float32, "fp64"),
                                         (torch.float64, "fp64")])
def test_fused_equals_levels_bitwise(dtype, arith):
    bt = W.shell_batch(m=40, nmin=3, nmax=5000, seed=11)
    a, _, _ = _run(bt, "levels", dtype, arith)
    b, _, _ = _run(bt, "fused", dtype, arith)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("order", ["caller", "tree"])
@pytest.mark.parametrize("products", ["both", "v", "w"])
def test_fused_orders_and_single_products(order, products):
    bt = W.shell_batch(m=25, nmin=20, nmax=3000, seed=12)
    a, _, _ = _run(bt, "levels", torch.float32, order=order, products=products)
    b, _, _ = _run(bt, "fused", torch.float32, order=order, products=products)
    if products != "w":
        assert torch.equal(a[0], b[0])
    if products != "v":
        assert torch.equal(a[1], b[1])


@pytest.mark.parametrize("host", [False, True])
def test_fused_graph_replay_and_host_buffers(host):
    bt = W.shell_batch(m=30, nmin=50, nmax=2500, seed=13)
    a, _, _ = _run(bt, "levels", torch.float32, host=host)
    b, _, _ = _run(bt, "fused", torch.float32, host=host, graph=True, reps=4)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_fused_full_size_against_oracle():
    """The 2000-shell batch as benched (FP32 products, double-single build,
    replayed from the library's graph): every body against the FP64 oracle,
    and bit for bit against the level schedule."""
    bt = W.shell_batch(m=2000, nmin=50, nmax=5000, seed=0)
    b, v, w = _run(bt, "fused", torch.float32, graph=True, reps=3, seed=1000)
    a, _, _ = _run(bt, "levels", torch.float32, seed=1000)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    vr = torch.from_numpy(v).float().double().numpy()
    wr = torch.from_numpy(w).float().double().numpy()
    rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, W.interleave(*vr), wr)
    compare_per_body(b[0].double().numpy(), rq, bt.off, "res", 1e-5, "fused Q~v")
    compare_per_body(W.interleave(*b[1].double().numpy()), rqt, bt.off, "bead", 1e-5, "fused Q~^T w")


def test_fused_then_separate_products_need_transforms():
    zq = _zq()
    dev = _dev()
    bt = W.shell_batch(m=6, nmin=30, nmax=900, seed=14)
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    rng = np.random.default_rng(4)
    v = torch.from_numpy(rng.standard_normal((3, bt.N))).to(dev, torch.float32)
    qv = torch.empty(bt.n_residues, device=dev)
    ctx = zq.Context(0)
    ctx.set_step_schedule("fused")
    ctx.pipeline(bt.off, x, y, z, v, qv)
    with pytest.raises(zq.ZQError) as e:
        ctx.apply_Q(v)
    assert e.value.code == zq.ZQ_ESTATE
    ctx.build_transforms(x, y, z)  # makes the schedules the fused step skipped
    got = ctx.apply_Q(v)
    ctx.sync()
    assert torch.equal(got, qv)
    ctx.close()


def test_fused_falls_back_for_a_large_body():
    """A body over 8192 beads: the step runs on the level schedule and
    matches the oracle."""
    pts = [np.stack(W.ellipsoid_body(n=9000, seed=2).body(0), 1), np.stack(W.shell_body(300, seed=1).body(0), 1)]
    off = np.array([0, 9000, 9300], np.int64)
    P = np.concatenate(pts)
    bt = W.Batch(off, P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy())
    a, _, _ = _run(bt, "levels", torch.float64)
    b, v, w = _run(bt, "fused", torch.float64)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    rq, _ = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, W.interleave(*v), w)
    assert np.linalg.norm(b[0].numpy() - rq) <= 1e-12 * np.linalg.norm(rq)
