"""zq_get_residue_offsets on a context's tree.

- It must agree with zq_residue_offsets on the zq_get_tree arrays, in both
  row orders.
- It must raise before a tree exists.
- Q~v from the device, moved block by block from the in-order rows to the
  pre-order rows, must match the oracle's explicit Q~ (Algorithm 1) applied
  to v after that Q~ is reassembled by Sec. 3's recursion
  [Residue_p; diag(Q~_x, Q~_y)].  The tolerance is 1e-12 in FP64.
"""
import numpy as np
import pytest

import oracle
from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _recursive_layout(Qin, t, q):
    k = 3 * (int(t["left"][q] >= 0) + int(t["right"][q] >= 0))
    r0 = int(t["roff"][q])
    parts = [Qin[r0:r0 + k]]
    for child in (t["left"][q], t["right"][q]):
        if child >= 0:
            parts.append(_recursive_layout(Qin, t, int(child)))
    return np.vstack(parts)


def test_context_offsets_and_preorder_products():
    from paper_1708_08427_gb300 import zq

    dev = _dev()
    ctx = zq.Context(0)
    with pytest.raises(zq.ZQError):
        ctx.residue_offsets("preorder")
    bt = W.shell_batch(m=6, nmin=3, nmax=90, seed=11)
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx.build_tree_batched(bt.off, x, y, z)
    ctx.build_transforms(x, y, z)
    g = ctx.get_tree()
    offs = {}
    for order in ("inorder", "preorder"):
        node_off, body_off = ctx.residue_offsets(order)
        ref_node, ref_body = zq.residue_offsets(bt.off, g["left"], g["right"], order)
        np.testing.assert_array_equal(node_off, ref_node)
        np.testing.assert_array_equal(body_off, ref_body)
        offs[order] = node_off
    np.testing.assert_array_equal(offs["inorder"], g["roff"])
    rng = np.random.default_rng(4)
    v = rng.standard_normal((3, bt.N))
    qv = ctx.apply_Q(torch.from_numpy(v).to(dev)).cpu().numpy()
    ctx.sync()
    rows = 3 * ((g["left"] >= 0).astype(np.int64) + (g["right"] >= 0))
    qpre = np.empty_like(qv)
    for q in range(bt.N - bt.m):
        a, b = int(offs["inorder"][q]), int(offs["preorder"][q])
        qpre[b:b + rows[q]] = qv[a:a + rows[q]]
    for j in range(bt.m):
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        B = oracle.Body(*bt.body(j))
        Qin, _ = B.qgen()
        Qpre = _recursive_layout(Qin, B.tree(), B.tree()["root"])
        ref = Qpre @ W.interleave(v[0, o:o + n], v[1, o:o + n], v[2, o:o + n])
        r0 = 3 * o - 6 * j
        got = qpre[r0:r0 + 3 * n - 6]
        assert np.linalg.norm(got - ref) <= 1e-12 * max(np.linalg.norm(ref), 1.0), j
    ctx.close()
