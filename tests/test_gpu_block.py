"""Block form (k right-hand sides, rows of k values) against the FP64 oracle.

Every column of the block must equal the oracle's Q~v / Q~^T w of that
column: FP64 within 1e-12 and FP32 within 1e-5 relative per body and column
(the single-vector tolerances), by the body's 2-norm and element by element
(every element within tol * the body's largest |element|).  BF16 stores inputs and outputs in bfloat16
(8 significant bits) and computes in FP32: the reference is the oracle
applied to the bfloat16-rounded inputs, and the only other error is the
rounding of each output element to bfloat16 (8-bit significand, round to
nearest: relative error at most 2^-8)
plus FP32 arithmetic (~1e-6), so both per-body errors are held to
2^-8 + 1e-5.  Bodies span several segments and nodes above them
(n > 512), k is ragged (not a multiple of the warp width).
"""
import numpy as np
import pytest

import oracle
from _parity import compare_per_body
from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5, torch.bfloat16: 2.0 ** -8 + 1e-5}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _ctx(bt):
    from paper_1708_08427_gb300 import zq

    dev = _dev()
    x, y, z = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(0)
    ctx.build_tree_batched(bt.off, x, y, z, 0)
    ctx.build_transforms(x, y, z)
    return ctx


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("k", [1, 7, 64])
def test_block_form_matches_oracle(dtype, k):
    bt = W.shell_batch(m=5, nmin=40, nmax=1500, seed=7)
    ctx = _ctx(bt)
    dev = _dev()
    rng = np.random.default_rng(100 + k)
    V = torch.from_numpy(rng.standard_normal((3 * bt.N, k))).to(dev, dtype)
    Wr = torch.from_numpy(rng.standard_normal((bt.n_residues, k))).to(dev, dtype)
    ctx.reserve_block(k, dtype)
    QV = ctx.apply_Q_block(V).double().cpu().numpy()
    QTW = ctx.apply_QT_block(Wr).double().cpu().numpy()
    ctx.sync()
    Vd = V.double().cpu().numpy()   # the (rounded) inputs the kernel saw
    Wd = Wr.double().cpu().numpy()
    for c in range(k):
        rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, W.interleave(*Vd[:, c].reshape(3, bt.N)), Wd[:, c])
        compare_per_body(QV[:, c], rq, bt.off, "res", TOL[dtype], f"{dtype} k={k} Q~V column {c}")
        compare_per_body(W.interleave(*QTW[:, c].reshape(3, bt.N)), rqt, bt.off, "bead", TOL[dtype],
                         f"{dtype} k={k} Q~^T W column {c}")
    ctx.close()


# unit roundoff of the tensor-core operands: TF32 keeps 11 significant bits,
# bfloat16 8
TC_U = {torch.float32: 2.0 ** -11, torch.bfloat16: 2.0 ** -8}


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("k", [1, 7, 64])
def test_block_form_tensor_cores_within_rounding_bound(dtype, k):
    """ZQ_TF32 / ZQ_BF16_TC: each node's G and input block are rounded once
    to the tensor-core type (relative u), so one node step errs by at most
    (|dG| + |du|) |u_p| <= (3 + 1) u |u_p| (|G|_F <= 3 for k_p <= 9);
    the steps of one height act on disjoint subtrees and the errors of lower
    heights pass through orthogonal maps without growth, so a body of height
    H errs by at most 4 H u |v| (+ u for bfloat16 output rounding).  Held per
    body against the oracle on the rounded inputs; the measured error is
    reported (print) and is far below this first-order bound."""
    bt = W.shell_batch(m=5, nmin=40, nmax=1500, seed=7)
    ctx = _ctx(bt)
    dev = _dev()
    rng = np.random.default_rng(300 + k)
    V = torch.from_numpy(rng.standard_normal((3 * bt.N, k))).to(dev, dtype)
    Wr = torch.from_numpy(rng.standard_normal((bt.n_residues, k))).to(dev, dtype)
    ctx.reserve_block(k, dtype)
    QV = ctx.apply_Q_block(V, tensor_cores=True).double().cpu().numpy()
    QTW = ctx.apply_QT_block(Wr, tensor_cores=True).double().cpu().numpy()
    ctx.sync()
    Vd = V.double().cpu().numpy()
    Wd = Wr.double().cpu().numpy()
    u = TC_U[dtype]
    H = [int(oracle.Body(*bt.body(j)).tree()["height"].max()) for j in range(bt.m)]
    worst = 0.0
    for c in range(k):
        rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, W.interleave(*Vd[:, c].reshape(3, bt.N)), Wd[:, c])
        got_t = W.interleave(*QTW[:, c].reshape(3, bt.N))
        ro = 0
        for j in range(bt.m):
            o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
            bound = (4 * H[j] + 1) * u
            e1 = np.linalg.norm(QV[ro:ro + 3 * n - 6, c] - rq[ro:ro + 3 * n - 6]) / np.linalg.norm(
                Vd[:, c].reshape(3, bt.N)[:, o:o + n])
            e2 = np.linalg.norm(got_t[3 * o:3 * (o + n)] - rqt[3 * o:3 * (o + n)]) / np.linalg.norm(
                Wd[ro:ro + 3 * n - 6, c])
            assert e1 <= bound and e2 <= bound, (j, H[j], e1, e2, bound)
            worst = max(worst, e1, e2)
            ro += 3 * n - 6
    print(f"tensor-core block form {dtype} k={k}: worst relative error {worst:.2e}")
    ctx.close()


def test_block_form_equals_single_column_path():
    """FP32: each column of the block form equals the column-major apply of
    that column (same transforms, same arithmetic per column)."""
    bt = W.shell_batch(m=4, nmin=100, nmax=900, seed=3)
    ctx = _ctx(bt)
    dev = _dev()
    k = 9
    rng = np.random.default_rng(5)
    V = torch.from_numpy(rng.standard_normal((3 * bt.N, k))).to(dev, torch.float32)
    ctx.reserve_block(k, torch.float32)
    QV = ctx.apply_Q_block(V)
    cols = ctx.apply_Q(V.t().contiguous().reshape(k, 3, bt.N))
    ctx.sync()
    np.testing.assert_allclose(QV.t().cpu().numpy(), cols.cpu().numpy(), rtol=0, atol=1e-6)
    ctx.close()


def test_block_form_needs_reservation():
    from paper_1708_08427_gb300 import zq

    bt = W.shell_batch(m=2, nmin=50, nmax=80, seed=1)
    ctx = _ctx(bt)
    dev = _dev()
    V = torch.zeros((3 * bt.N, 4), device=dev)
    with pytest.raises(zq.ZQError) as e:
        ctx.apply_Q_block(V)
    assert e.value.code == zq.ZQ_ESTATE
    ctx.reserve_block(2, torch.float32)
    with pytest.raises(zq.ZQError) as e:
        ctx.apply_Q_block(V)  # k = 4 > reserved 2
    assert e.value.code == zq.ZQ_ESTATE
    ctx.close()
