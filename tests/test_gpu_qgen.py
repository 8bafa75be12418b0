"""The explicit Q~ in CSR form (zq_qgen, Algorithm 1) against the oracle.

Small bodies: the CSR structure is bit-exact against the oracle's tree (row
lengths 3 n_p for node p's rows; the columns of a row are p's beads in tree
order, three axes each, as 3 perm[pos] + a), and the values match the
oracle's dense Q~ and U (Q_Z's rotational rows) per body, FP64 within
1e-12 and FP32 within 1e-5 relative (Frobenius norm per body, and every
entry within tol * the body's largest |entry|).

At a larger size, where the oracle's dense form would not fit, properties
that hold at any size: the CSR Q~ times v equals zq_apply_Q(v) and its
transpose times w equals zq_apply_QT(w) (1e-12 FP64 relative), every row
has unit norm, and U v is the rotational half of the root Info-set that
zq_apply_Q_full returns.
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


def _ctx(bt):
    from paper_1708_08427_gb300 import zq

    dev = _dev()
    x, y, z = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(0)
    ctx.build_tree_batched(bt.off, x, y, z)
    ctx.build_transforms(x, y, z)
    return ctx


def _small_batch():
    bt = W.shell_batch(m=6, nmin=20, nmax=700, seed=71)
    rng = np.random.default_rng(4)
    pts = [np.stack(bt.body(j), 1) for j in range(bt.m)]
    pts.append(rng.uniform(-1, 1, (3, 3)))                                  # smallest body
    pts.append(np.c_[rng.uniform(-1, 1, (40, 2)), np.full(40, 0.3)])        # flat
    off = np.zeros(len(pts) + 1, np.int64)
    off[1:] = np.cumsum([p.shape[0] for p in pts])
    P = np.concatenate(pts)
    return W.Batch(off, P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy())


@pytest.fixture(scope="module")
def small():
    bt = _small_batch()
    ctx = _ctx(bt)
    bodies = [oracle.Body(*bt.body(j)) for j in range(bt.m)]
    yield ctx, bt, bodies
    ctx.close()


def test_structure_is_the_tree(small):
    ctx, bt, bodies = small
    rp, col, val, _ = ctx.qgen(torch.float64)
    rp, col = rp.cpu().numpy(), col.cpu().numpy()
    assert rp[0] == 0 and rp[-1] == col.shape[0] == ctx.qgen_nnz()
    rbase = 0
    for j, B in enumerate(bodies):
        o = int(bt.off[j])
        t = B.tree()
        for g in range(B.n - 1):
            k = B.node(g)["k"]
            if k == 3:
                continue
            pos = np.arange(t["first"][g], t["last"][g] + 1)
            want = (3 * (o + t["perm"][pos])[:, None] + np.arange(3)).reshape(-1)
            for i in range(k - 3):
                r = rbase + int(t["roff"][g]) + i
                np.testing.assert_array_equal(col[rp[r]:rp[r + 1]], want)
        rbase += 3 * B.n - 6


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_values_match_dense_oracle(small, dtype, tol):
    ctx, bt, bodies = small
    rp, col, val, U = ctx.qgen(dtype, with_u=True)
    rp, col = rp.cpu().numpy(), col.cpu().numpy()
    val, U = val.double().cpu().numpy(), U.double().cpu().numpy()
    worst = 0.0
    rbase = 0
    for j, B in enumerate(bodies):
        o, n = int(bt.off[j]), B.n
        Qt, QZ = B.qgen()
        D = np.zeros((3 * n - 6, 3 * n))
        for r in range(3 * n - 6):
            a, b = rp[rbase + r], rp[rbase + r + 1]
            D[r, col[a:b] - 3 * o] = val[a:b]
        rbase += 3 * n - 6
        worst = max(worst, np.linalg.norm(D - Qt) / np.linalg.norm(Qt), np.abs(D - Qt).max() / np.abs(Qt).max())
        Uj = U[9 * o:9 * (o + n)].reshape(3, 3 * n)
        worst = max(worst, np.linalg.norm(Uj - QZ[3:]) / np.linalg.norm(QZ[3:]),
                    np.abs(Uj - QZ[3:]).max() / np.abs(QZ[3:]).max())
    assert worst <= tol, worst


def test_large_batch_properties():
    bt = W.shell_batch(m=120, nmin=50, nmax=5000, seed=73)
    ctx = _ctx(bt)
    dev = _dev()
    N, R = bt.N, bt.n_residues
    rp, col, val, U = ctx.qgen(torch.float64, with_u=True)
    rows = torch.repeat_interleave(torch.arange(R, device=dev), rp[1:] - rp[:-1])
    col = col.long()
    g = torch.Generator(device="cpu").manual_seed(5)
    v = torch.randn((3, N), generator=g, dtype=torch.float64).to(dev)
    w = torch.randn(R, generator=g, dtype=torch.float64).to(dev)
    vi = v.t().reshape(-1)                                          # interleaved: 3 i + a
    qv = torch.zeros(R, dtype=torch.float64, device=dev).index_add_(0, rows, val * vi[col])
    qtw = torch.zeros(3 * N, dtype=torch.float64, device=dev).index_add_(0, col, val * w[rows])
    ref_qv, root = ctx.apply_Q_full(v)
    ref_qtw = ctx.apply_QT(w)
    norms = torch.zeros(R, dtype=torch.float64, device=dev).index_add_(0, rows, val * val)
    body = torch.repeat_interleave(torch.arange(bt.m, device=dev), torch.from_numpy(np.diff(bt.off)).to(dev))
    off = torch.from_numpy(bt.off).to(dev)
    nj = (off[1:] - off[:-1])[body]
    loc = torch.arange(N, device=dev) - off[:-1][body]
    Uv = torch.zeros((bt.m, 3), dtype=torch.float64, device=dev)
    for e in range(3):
        # U_j[e, 3 i + a] sits at 9 off_j + e 3 n_j + 3 i + a
        idx = 9 * off[:-1][body] + e * 3 * nj + 3 * loc
        part = sum(U[idx + a] * v[a] for a in range(3))
        Uv[:, e].index_add_(0, body, part)
    ctx.sync()
    e1 = ((qv - ref_qv).norm() / ref_qv.norm()).item()
    e2 = ((qtw.view(N, 3).t() - ref_qtw).norm() / ref_qtw.norm()).item()
    e3 = (norms - 1).abs().max().item()
    e4 = ((Uv - root[:, 3:]).norm() / root[:, 3:].norm()).item()
    assert max(e1, e2, e3, e4) <= 1e-12, (e1, e2, e3, e4)
    ctx.close()


def test_large_body_path_properties():
    """One body of 20,000 beads (the device-wide tree path, thousands of
    nodes above the segments) next to small ones: CSR Q~ v equals
    zq_apply_Q in FP64 and FP32, every row has unit norm."""
    big = W.ellipsoid_body(n=20000, seed=5)
    small = W.shell_batch(m=3, nmin=40, nmax=600, seed=6)
    pts = [np.stack(big.body(0), 1)] + [np.stack(small.body(j), 1) for j in range(small.m)]
    off = np.zeros(len(pts) + 1, np.int64)
    off[1:] = np.cumsum([p.shape[0] for p in pts])
    P = np.concatenate(pts)
    bt = W.Batch(off, P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy())
    ctx = _ctx(bt)
    dev = _dev()
    N, R = bt.N, bt.n_residues
    g = torch.Generator(device="cpu").manual_seed(7)
    v64 = torch.randn((3, N), generator=g, dtype=torch.float64).to(dev)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        rp, col, val, _ = ctx.qgen(dt)
        rows = torch.repeat_interleave(torch.arange(R, device=dev), rp[1:] - rp[:-1])
        v = v64.to(dt)
        vi = v.t().reshape(-1)
        qv = torch.zeros(R, dtype=dt, device=dev).index_add_(0, rows, val * vi[col.long()])
        ref = ctx.apply_Q(v)
        norms = torch.zeros(R, dtype=torch.float64, device=dev).index_add_(0, rows, val.double() ** 2)
        ctx.sync()
        e1 = ((qv - ref).double().norm() / ref.double().norm()).item()
        e2 = (norms - 1).abs().max().item()
        assert e1 <= tol and e2 <= 10 * tol, (dt, e1, e2)
    ctx.close()
