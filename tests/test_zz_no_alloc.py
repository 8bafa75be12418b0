"""zq_apply_Q_noalloc: Q~v for one body with its intermediates in the
library's static device array, no allocation in the call.

Checked against the context path (zq_build_tree + zq_build_transforms +
zq_apply_Q, FP64) and against the FP64 oracle directly, within the FP64
parity tolerance (by norm and element by element), on consecutive calls
that reuse the one static array with different body sizes.  The argument
checks run without a GPU.
"""
import ctypes

import numpy as np
import pytest

import oracle
from _parity import compare_elementwise
from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")

TOL = 1e-12


def _lib():
    from paper_1708_08427_gb300 import zq

    return zq, zq._lib()


def test_noalloc_rejects_bad_arguments_without_gpu():
    zq, L = _lib()
    buf = ctypes.c_double * 16
    a = buf()
    p = ctypes.addressof(a)
    for n in (0, 2, zq.ZQ_NOALLOC_MAX_BEADS + 1, 1 << 40):
        assert L.zq_apply_Q_noalloc(0, None, n, p, p, p, p, p) == zq.ZQ_EINVAL
    assert L.zq_apply_Q_noalloc(0, None, 8, None, p, p, p, p) == zq.ZQ_EINVAL
    assert L.zq_apply_Q_noalloc(0, None, 8, p, p, p, p, None) == zq.ZQ_EINVAL
    assert L.zq_apply_Q_noalloc(-1, None, 8, p, p, p, p, p) == zq.ZQ_EINVAL
    with pytest.raises(ValueError, match="beads"):
        zq.apply_Q_noalloc(torch.zeros(2, dtype=torch.float64), None, None, None, None)


def _reference(bt, dev, v):
    zq, _ = _lib()
    x, y, z = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(0)
    ctx.build_tree(x, y, z)
    ctx.build_transforms(x, y, z)
    ref = ctx.apply_Q(v).cpu().numpy()
    ctx.sync(allow_degenerate=True)
    ctx.close()
    return x, y, z, ref


@pytest.mark.gpu
def test_noalloc_matches_context_path_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    zq, _ = _lib()
    dev = torch.device("cuda:0")
    cases = []
    for n, seed in ((zq.ZQ_NOALLOC_MAX_BEADS, 1), (701, 2), (3, 3), (1500, 4)):
        bt = W.shell_body(n=n, seed=seed)
        v = torch.from_numpy(W.vectors(10 + seed, 3 * n).reshape(3, n)).to(dev)
        x, y, z, ref = _reference(bt, dev, v)
        cases.append((n, x, y, z, v, ref))
    # two calls in a row on the same body, then the other sizes, then the
    # first body again: each call must leave nothing behind for the next
    order = [0, 0, 1, 2, 3, 0]
    outs = []
    for i in order:
        n, x, y, z, v, ref = cases[i]
        out = torch.full((3 * n - 6,), float("nan"), dtype=torch.float64, device=dev)
        zq.apply_Q_noalloc(x, y, z, v, out)
        outs.append(out)
    torch.cuda.synchronize()
    for i, out in zip(order, outs):
        n, x, y, z, v, ref = cases[i]
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), n
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err <= TOL, (n, err)
        # and against the oracle itself, element by element
        B = oracle.Body(x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy())
        want = B.apply_Q(W.interleave(*v.cpu().numpy()))
        compare_elementwise(got, want, TOL, f"n = {n}")
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[5])
