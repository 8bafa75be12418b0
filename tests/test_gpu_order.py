"""Tree-ordered bead vectors (zq_set_vector_order): the products take and
give the bead planes in the tree's sorted-position order, skipping the
gather through the permutation.  They must be the caller-order results
permuted, bit for bit (the same numbers enter the same arithmetic): single
columns in FP32 and FP64, both products at once, the k-column block form,
and the whole step with the tree kept."""
import numpy as np
import pytest

from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_tree_order_is_the_permuted_caller_order():
    from paper_1708_08427_gb300 import zq

    dev = _dev()
    bt = W.shell_batch(m=12, nmin=30, nmax=2500, seed=77)
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(0)
    ctx.build_tree_batched(bt.off, x, y, z)
    ctx.build_transforms(x, y, z)
    perm = torch.from_numpy(ctx.get_tree()["perm"].astype(np.int64)).to(dev)
    rng = np.random.default_rng(3)
    for dt in (torch.float32, torch.float64):
        v = torch.from_numpy(rng.standard_normal((3, bt.N))).to(dev, dt)
        w = torch.from_numpy(rng.standard_normal(bt.n_residues)).to(dev, dt)
        ctx.set_vector_order("caller")
        q1, t1 = ctx.apply_Q(v), ctx.apply_QT(w)
        p1, pt1 = ctx.apply_pair(v, w)
        ctx.set_vector_order("tree")
        vt = v[:, perm].contiguous()
        q2, t2 = ctx.apply_Q(vt), ctx.apply_QT(w)
        p2, pt2 = ctx.apply_pair(vt, w)
        ctx.sync()
        assert torch.equal(q1, q2) and torch.equal(p1, p2)
        assert torch.equal(t1[:, perm], t2) and torch.equal(pt1[:, perm], pt2)
    # block form, 5 columns
    k = 5
    V = torch.from_numpy(rng.standard_normal((3 * bt.N, k))).to(dev, torch.float32)
    Wr = torch.from_numpy(rng.standard_normal((bt.n_residues, k))).to(dev, torch.float32)
    ctx.reserve_block(k, torch.float32)
    ctx.set_vector_order("caller")
    B1, C1 = ctx.apply_Q_block(V), ctx.apply_QT_block(Wr)
    ctx.set_vector_order("tree")
    Vt = V.view(3, bt.N, k)[:, perm].reshape(3 * bt.N, k).contiguous()
    B2, C2 = ctx.apply_Q_block(Vt), ctx.apply_QT_block(Wr)
    ctx.sync()
    assert torch.equal(B1, B2)
    assert torch.equal(C1.view(3, bt.N, k)[:, perm], C2.view(3, bt.N, k))
    # the whole step with the tree kept
    v = torch.from_numpy(rng.standard_normal((3, bt.N))).to(dev, torch.float32)
    w = torch.from_numpy(rng.standard_normal(bt.n_residues)).to(dev, torch.float32)
    qv1, qt1 = torch.empty(bt.n_residues, device=dev), torch.empty((3, bt.N), device=dev)
    qv2, qt2 = torch.empty_like(qv1), torch.empty_like(qt1)
    ctx.set_vector_order("caller")
    ctx.pipeline(bt.off, x, y, z, v, qv1, w, qt1, keep_tree=True)
    ctx.set_vector_order("tree")
    ctx.pipeline(bt.off, x, y, z, v[:, perm].contiguous(), qv2, w, qt2, keep_tree=True)
    ctx.sync()
    assert torch.equal(qv1, qv2) and torch.equal(qt1[:, perm], qt2)
    ctx.close()
