"""The GPU parity tests' helpers, checked on the CPU.

residue_scales gives each residue of Q~v the 2-norm of the bead vectors
below its node.  Orthogonality of the node transforms (Sec. 3) bounds every
residue by that norm, and the root's residues get the whole body's norm.
record_to_G turns the library's record layout back into G; checked here on
a record built from a known product of reflectors."""
import numpy as np

import oracle
from _parity import compare_per_body, errors_per_body, record_to_G, residue_scales
from paper_1708_08427_gb300 import workloads as W


def test_residue_scales_bound_every_residue():
    bt = W.shell_batch(m=6, nmin=3, nmax=400, seed=3)
    rng = np.random.default_rng(0)
    f = rng.standard_normal(3 * bt.N)
    rq, _ = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, f, np.zeros(bt.n_residues))
    s = residue_scales(bt.off, bt.x, bt.y, bt.z, f)
    assert s.shape == rq.shape
    assert np.all(np.abs(rq) <= s * (1 + 1e-12))
    # the root of each body sees all of the body's beads
    for j in range(bt.m):
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        B = oracle.Body(*bt.body(j))
        t = B.tree()
        r0 = 3 * o - 6 * j + int(t["roff"][t["root"]])
        assert np.isclose(s[r0], np.linalg.norm(f[3 * o:3 * (o + n)]))


def test_elementwise_check_catches_one_wrong_element():
    bt = W.shell_batch(m=3, nmin=200, nmax=300, seed=1)
    rng = np.random.default_rng(2)
    ref = rng.standard_normal(bt.n_residues)
    got = ref.copy()
    got[17] += 5 * 1e-5 * np.abs(ref[:3 * int(bt.off[1]) - 6]).max()
    ne, ee = errors_per_body(got, ref, bt.off, "res")
    assert ne[0] < 1e-5 < ee[0]  # hidden in the norm, caught element by element
    try:
        compare_per_body(got, ref, bt.off, "res", 1e-5)
    except AssertionError:
        return
    raise AssertionError("a wrong element passed")


def test_record_to_G_expands_reflectors():
    rng = np.random.default_rng(4)
    for k in (6, 9):
        M = rng.standard_normal((3, k))
        L, G = oracle.lq(M)
        # the compact record of this G: Householder vectors of M^T's QR
        A = M.T.copy()
        rec = np.zeros(28)
        tail = 5
        Gr = np.eye(k)
        for j in range(3):
            x = A[j:, j]
            a = x[0]
            nrm = np.linalg.norm(x)
            b = -nrm if a >= 0 else nrm
            tau = (b - a) / b
            v = np.zeros(k)
            v[j] = 1.0
            v[j + 1:] = x[1:] / (a - b)
            A = A - tau * np.outer(v, v @ A)
            Gr = Gr - tau * np.outer(v, v @ Gr)
            rec[2 + j] = tau
            rec[tail:tail + k - 1 - j] = v[j + 1:]
            tail += k - 1 - j
        for j in range(3):
            if A[j, j] < 0:
                rec[2 + j] = -rec[2 + j]
        np.testing.assert_allclose(record_to_G(rec, k), G, atol=1e-13)
