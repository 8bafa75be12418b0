"""zq_residue_offsets (host only, no GPU): each node's residue rows in the
two row orders of Q~ (Sec. 3).

- In-order, the order of every product, must be the oracle's residue
  offsets.
- Pre-order must give the paper's recursive layout
  Q~_p = [Residue_p; diag(Q~_x, Q~_y)].  This is checked on the oracle's
  explicit Q~ (Algorithm 1).  Its rows, moved to the pre-order offsets,
  must equal a direct recursive assembly of that formula.  Every subtree's
  rows must then form one contiguous block whose nonzero columns are the
  subtree's own beads.
- A hand-worked 5-bead tree pins both orders.
- Malformed trees are rejected.
"""
import numpy as np
import pytest

import oracle
from paper_1708_08427_gb300 import workloads as W


@pytest.fixture(scope="module")
def zq():
    from paper_1708_08427_gb300 import build

    build.build()
    from paper_1708_08427_gb300 import zq as mod

    return mod


def test_hand_worked_five_bead_tree(zq):
    # sorted beads 0..4; root (id 1) splits {0,1} | {2,3,4}; node 0 = (0, 1);
    # node 3 = (node 2, bead 4); node 2 = (2, 3).  Rows: 3 per internal child,
    # so node 1 has 6, node 3 has 3, nodes 0 and 2 none (3 * 5 - 6 = 9).
    off = [0, 5]
    left = [-1, 0, -3, 2]
    right = [-2, 3, -4, -5]
    ino, body = zq.residue_offsets(off, left, right, "inorder")
    pre, _ = zq.residue_offsets(off, left, right, "preorder")
    np.testing.assert_array_equal(ino, [0, 0, 6, 6])  # by id: 0 | 6 | 0 | 3 rows
    np.testing.assert_array_equal(pre, [6, 0, 9, 6])  # root, left subtree, node 3, node 2
    np.testing.assert_array_equal(body, [0, 9])


def _global_tree(bt, bodies):
    """The oracle's trees in zq_get_tree's global numbering."""
    nodes = bt.N - bt.m
    left = np.empty(nodes, np.int32)
    right = np.empty(nodes, np.int32)
    roff = np.empty(nodes, np.int64)
    trees = []
    rbase = 0
    for j, B in enumerate(bodies):
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        nb = o - j
        t = B.tree()
        trees.append(t)

        def glob(code):
            return np.where(code >= 0, code + nb, -1 - (o + (-1 - code)))

        left[nb:nb + n - 1] = glob(t["left"])
        right[nb:nb + n - 1] = glob(t["right"])
        roff[nb:nb + n - 1] = t["roff"] + rbase
        rbase += 3 * n - 6
    return left, right, roff, trees


def _recursive_layout(Qin, t, q):
    """Sec. 3's Q~_q = [Residue_q; diag(Q~_x, Q~_y)] over the body's global
    columns: the node's own rows (its block of the in-order Q~), then the
    left subtree's rows, then the right subtree's (columns of the two
    subtrees are disjoint, so diag(.,.) stacks them)."""
    k = 3 * (int(t["left"][q] >= 0) + int(t["right"][q] >= 0))
    r0 = int(t["roff"][q])
    parts = [Qin[r0:r0 + k]]
    for child in (t["left"][q], t["right"][q]):
        if child >= 0:
            parts.append(_recursive_layout(Qin, t, int(child)))
    return np.vstack(parts)


@pytest.mark.parametrize("seed", [0, 1])
def test_orders_against_the_oracle(zq, seed):
    bt = W.shell_batch(m=5, nmin=3, nmax=70, seed=seed)
    bodies = [oracle.Body(*bt.body(j)) for j in range(bt.m)]
    left, right, roff, trees = _global_tree(bt, bodies)
    ino, body = zq.residue_offsets(bt.off, left, right, "inorder")
    pre, body2 = zq.residue_offsets(bt.off, left, right, "preorder")
    np.testing.assert_array_equal(ino, roff)
    np.testing.assert_array_equal(body, body2)
    np.testing.assert_array_equal(body, 3 * bt.off - 6 * np.arange(bt.m + 1))
    for j, (B, t) in enumerate(zip(bodies, trees)):
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        nb, rb = o - j, int(body[j])
        Qin, _ = B.qgen()
        Qpre = np.zeros_like(Qin)
        for g in range(n - 1):
            k = 3 * (int(t["left"][g] >= 0) + int(t["right"][g] >= 0))
            Qpre[pre[nb + g] - rb:pre[nb + g] - rb + k] = Qin[roff[nb + g] - rb:roff[nb + g] - rb + k]
        np.testing.assert_array_equal(Qpre, _recursive_layout(Qin, t, t["root"]))
        # each subtree: one contiguous row block, nonzero only on its own beads
        for g in range(n - 1):
            cnt = int(t["last"][g] - t["first"][g] + 1)
            r0 = int(pre[nb + g] - rb)
            block = Qpre[r0:r0 + 3 * cnt - 6]
            own = np.zeros(3 * n, bool)
            for s in range(int(t["first"][g]), int(t["last"][g]) + 1):
                i = int(t["perm"][s])
                own[3 * i:3 * i + 3] = True
            assert not np.any(block[:, ~own]), (j, g)
            assert np.linalg.matrix_rank(block) == block.shape[0]


def test_malformed_trees_are_rejected(zq):
    off = [0, 5]
    good = ([-1, 0, -3, 2], [-2, 3, -4, -5])
    zq.residue_offsets(off, *good)
    bad = [
        ([-1, 0, -3, 2], [-2, 3, -4, -6]),  # a leaf outside the body
        ([-1, 0, -3, 2], [-2, 4, -4, -5]),  # an internal child outside the body
        ([-1, 0, -3, 0], [-2, 3, -4, -5]),  # node 0 the child of two nodes
        ([-1, 0, 3, 2], [-2, -5, -4, -3]),  # nodes 2 and 3 a cycle, not reached from the root
        ([-1, 1, -3, 2], [-2, 3, -4, -5]),  # a node its own child
    ]
    for left, right in bad:
        for order in ("inorder", "preorder"):
            with pytest.raises(zq.ZQError):
                zq.residue_offsets(off, left, right, order)
    with pytest.raises(zq.ZQError):  # a body of two beads
        zq.residue_offsets([0, 2, 7], [-1] * 5, [-2] * 5, "inorder")
    n = np.empty(4, np.int64)
    lf, rt = (np.ascontiguousarray(a, np.int32) for a in good)
    offa = np.array(off, np.int64)
    args = (1, offa.ctypes.data_as(zq._i64p), zq._np_i32(lf), zq._np_i32(rt))
    assert zq.zq_residue_offsets(*args, 2, n.ctypes.data_as(zq._i64p), None) == zq.ZQ_EINVAL
    assert zq.zq_residue_offsets(*args, 1, None, None) == zq.ZQ_EINVAL
    assert zq.zq_residue_offsets(*args, 1, n.ctypes.data_as(zq._i64p), None) == zq.ZQ_OK
