"""The whole orthogonal Q = [Q_Z; Q~] (zq_apply_Q_full / zq_apply_QT_full):
the root Info-set Q_Z v of every body and the downward pass started from a
given root Velocity-set, against the FP64 oracle's root sets (Eq. 4.4,
Theorem 4.3), and the round trip Q_Z^T Q_Z v + Q~^T Q~ v = v.  Bodies both
below and above the segment size (roots inside a segment and among the
top nodes).  Every body's results are compared by norm and element by
element."""
import numpy as np
import pytest

import oracle
from _parity import compare_elementwise
from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_full_q_matches_oracle_and_round_trips(dtype):
    from paper_1708_08427_gb300 import zq

    dev = _dev()
    bt = W.shell_batch(m=14, nmin=3, nmax=3000, seed=41)
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(0)
    ctx.build_tree_batched(bt.off, x, y, z)
    ctx.build_transforms(x, y, z)
    rng = np.random.default_rng(6)
    v = rng.standard_normal((3, bt.N))
    w = rng.standard_normal(bt.n_residues)
    root_in = rng.standard_normal((bt.m, 6))
    tv = torch.from_numpy(v).to(dev, dtype)
    qv, root = ctx.apply_Q_full(tv)
    out = ctx.apply_QT_full(torch.from_numpy(w).to(dev, dtype), torch.from_numpy(root_in).to(dev, dtype))
    back = ctx.apply_QT_full(qv, root)
    ctx.sync()
    qv, root, out, back = (t.double().cpu().numpy() for t in (qv, root, out, back))
    tol = TOL[dtype]
    ro = 0
    for j in range(bt.m):
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        B = oracle.Body(*bt.body(j))
        f = W.interleave(*v[:, o:o + n])
        rq, r6 = B.apply_Q(f, with_root=True)
        compare_elementwise(qv[ro:ro + 3 * n - 6], rq, tol, f"body {j} residues")
        compare_elementwise(root[j], r6, tol, f"body {j} root Info-set")
        rqt = B.apply_QT(w[ro:ro + 3 * n - 6], root_in[j])
        compare_elementwise(W.interleave(*out[:, o:o + n]), rqt, tol, f"body {j} Q^T [r; w]")
        compare_elementwise(back[:, o:o + n], v[:, o:o + n], tol, f"body {j} round trip")
        ro += 3 * n - 6
    ctx.close()
