"""Products for rigidly moved bodies on kept transforms (zq_apply_rotated)
against the oracle's batch_apply_rotated: each bead vector rotated by R_j^T
into Q~, and each bead vector of Q~^T w rotated by R_j.  FP64 within 1e-12
and FP32 within 1e-5 relative per body.

The batch holds bodies of many segments, a body whose root (a node above
the segments) has a single far bead as a child (the leaf path of the
per-body top-node kernels), and the smallest body (3 beads, Case I at the
root).  R = I gives the plain products bit for bit, one product alone gives
the same bits as both at once, and Q~^T Q~ f on the moved bodies is the
moved bodies' projector f - Z^T (Z Z^T)^-1 Z f (basis-free, FP64 1e-12).
Products are compared per body by norm and element by element.
"""
import numpy as np
import pytest

import oracle
from _parity import compare_per_body
from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _rot(q):
    q0, q1, q2, q3 = q / np.linalg.norm(q)
    return np.array([[q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, 2 * (q1 * q2 - q0 * q3), 2 * (q1 * q3 + q0 * q2)],
                     [2 * (q1 * q2 + q0 * q3), q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3, 2 * (q2 * q3 - q0 * q1)],
                     [2 * (q1 * q3 - q0 * q2), 2 * (q2 * q3 + q0 * q1), q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3]])


def _batch():
    bt = W.shell_batch(m=9, nmin=20, nmax=2600, seed=61)
    rng = np.random.default_rng(6)
    pts = [np.stack(bt.body(j), 1) for j in range(bt.m)]
    sh = rng.standard_normal((1200, 3))
    sh = 3.0 * sh / np.linalg.norm(sh, axis=1, keepdims=True)
    pts.append(np.r_[sh, [[400.0, 0.0, 0.0]]])      # the root's second child is one far bead
    pts.append(rng.uniform(-1, 1, (3, 3)))           # the smallest body
    off = np.zeros(len(pts) + 1, np.int64)
    off[1:] = np.cumsum([p.shape[0] for p in pts])
    P = np.concatenate(pts)
    return W.Batch(off, P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy())


@pytest.fixture(scope="module")
def setup():
    from paper_1708_08427_gb300 import zq

    dev = _dev()
    bt = _batch()
    rng = np.random.default_rng(9)
    Rm = np.stack([_rot(rng.standard_normal(4)) for _ in range(bt.m)])
    x, y, z = (torch.from_numpy(a.copy()).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(0)
    ctx.build_tree_batched(bt.off, x, y, z)
    ctx.build_transforms(x, y, z)
    yield zq, ctx, bt, Rm, dev
    ctx.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_rotated_products_match_oracle(setup, dtype):
    zq, ctx, bt, Rm, dev = setup
    rng = np.random.default_rng(1)
    v = rng.standard_normal((3, bt.N))
    w = rng.standard_normal(bt.n_residues)
    R_d = torch.from_numpy(Rm.copy()).to(dev)
    qv, qtw = ctx.apply_rotated(R_d, torch.from_numpy(v).to(dev, dtype), torch.from_numpy(w).to(dev, dtype))
    ctx.sync()
    rq, rqt = oracle.batch_apply_rotated(bt.off, bt.x, bt.y, bt.z, Rm, W.interleave(*v), w)
    compare_per_body(qv.double().cpu().numpy(), rq, bt.off, "res", TOL[dtype], "rotated Q~v")
    compare_per_body(W.interleave(*qtw.double().cpu().numpy()), rqt, bt.off, "bead", TOL[dtype], "rotated Q~^T w")


def test_identity_rotation_and_single_products(setup):
    zq, ctx, bt, Rm, dev = setup
    rng = np.random.default_rng(2)
    for dt in (torch.float32, torch.float64):
        v = torch.from_numpy(rng.standard_normal((3, bt.N))).to(dev, dt)
        w = torch.from_numpy(rng.standard_normal(bt.n_residues)).to(dev, dt)
        eye = torch.eye(3, dtype=torch.float64, device=dev).repeat(bt.m, 1, 1).contiguous()
        a = ctx.apply_rotated(eye, v, w)
        b = ctx.apply_pair(v, w)
        R_d = torch.from_numpy(Rm.copy()).to(dev)
        both = ctx.apply_rotated(R_d, v, w)
        only_v, _ = ctx.apply_rotated(R_d, v=v)
        _, only_w = ctx.apply_rotated(R_d, w=w)
        ctx.sync()
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
        assert torch.equal(both[0], only_v) and torch.equal(both[1], only_w)


def test_projector_of_the_moved_bodies(setup):
    zq, ctx, bt, Rm, dev = setup
    rng = np.random.default_rng(3)
    P = np.stack([bt.x, bt.y, bt.z], 1)
    f = rng.standard_normal((bt.N, 3))
    R_d = torch.from_numpy(Rm.copy()).to(dev)
    qf, _ = ctx.apply_rotated(R_d, v=torch.from_numpy(f.T.copy()).to(dev))
    _, pf = ctx.apply_rotated(R_d, w=qf)
    ctx.sync()
    got = pf.cpu().numpy().T
    worst = 0.0
    for j in range(bt.m):
        a, b = int(bt.off[j]), int(bt.off[j + 1])
        p = P[a:b] @ Rm[j].T                           # the moved body (translation irrelevant)
        p = p - p.mean(0)
        g = f[a:b]
        J = (p * p).sum() * np.eye(3) - p.T @ p
        om = np.linalg.solve(J, np.cross(p, g).sum(0))
        want = g - (g.mean(0) + np.cross(om, p))
        worst = max(worst, np.linalg.norm(got[a:b] - want) / np.linalg.norm(g))
    assert worst <= 1e-12, worst
