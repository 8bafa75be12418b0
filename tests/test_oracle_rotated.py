"""Pins of the oracle's products for rigidly moved bodies (batch_apply_rotated).

The products are taken on the transforms of the reference coordinates with
every bead vector rotated by R_j^T on the way in and R_j on the way out.
They are checked against what fixes them without reference to the
transforms: the moved body's own Z (Eq. 1.2, built here from the moved
coordinates) must annihilate Q~^T w, Q~^T must be an isometry, and
Q~^T Q~ must be the moved body's orthogonal projector
I - Z^T (Z Z^T)^-1 Z (Z of the centred moved beads, which has the same row
space: a translation adds multiples of the force rows to the torque rows).  Passing R_j instead of R_j^T (a transposed
rotation, the plausible mistake) must fail the annihilation check.
"""
import numpy as np
import pytest

import oracle
from paper_1708_08427_gb300 import workloads as W


def _rot(q):
    q0, q1, q2, q3 = q / np.linalg.norm(q)
    return np.array([[q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3, 2 * (q1 * q2 - q0 * q3), 2 * (q1 * q3 + q0 * q2)],
                     [2 * (q1 * q2 + q0 * q3), q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3, 2 * (q2 * q3 - q0 * q1)],
                     [2 * (q1 * q3 - q0 * q2), 2 * (q2 * q3 + q0 * q1), q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3]])


def _moved(bt, seed):
    rng = np.random.default_rng(seed)
    Rm = np.stack([_rot(rng.standard_normal(4)) for _ in range(bt.m)])
    P = np.stack([bt.x, bt.y, bt.z], 1)
    Pm = P.copy()
    for j in range(bt.m):
        a, b = bt.off[j], bt.off[j + 1]
        Pm[a:b] = P[a:b] @ Rm[j].T + rng.standard_normal(3) * 5.0
    return Rm, Pm


def _Z(P):
    """6 x 3n: rows 0-2 sum the bead vectors, rows 3-5 sum r_k x f_k (Eq. 1.2)."""
    n = P.shape[0]
    Z = np.zeros((6, 3 * n))
    for k in range(n):
        Z[0:3, 3 * k:3 * k + 3] = np.eye(3)
        x, y, z = P[k]
        Z[3:6, 3 * k:3 * k + 3] = np.array([[0, -z, y], [z, 0, -x], [-y, x, 0]])
    return Z


@pytest.fixture(scope="module")
def case():
    bt = W.shell_batch(m=5, nmin=7, nmax=90, seed=41)
    Rm, Pm = _moved(bt, 3)
    return bt, Rm, Pm


def test_identity_rotation_is_the_plain_product(case):
    bt, _, _ = case
    rng = np.random.default_rng(1)
    f = rng.standard_normal(3 * bt.N)
    w = rng.standard_normal(bt.n_residues)
    I = np.tile(np.eye(3), (bt.m, 1, 1))
    a = oracle.batch_apply_rotated(bt.off, bt.x, bt.y, bt.z, I, f, w)
    b = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, f, w)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _checks(bt, Rm, Pm, seed):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(bt.n_residues)
    f = rng.standard_normal(3 * bt.N)
    _, qtw = oracle.batch_apply_rotated(bt.off, bt.x, bt.y, bt.z, Rm, None, w)
    qf, _ = oracle.batch_apply_rotated(bt.off, bt.x, bt.y, bt.z, Rm, f, None)
    _, pf = oracle.batch_apply_rotated(bt.off, bt.x, bt.y, bt.z, Rm, None, qf)
    ann, iso, proj = 0.0, 0.0, 0.0
    ro = 0
    for j in range(bt.m):
        a, b = int(bt.off[j]), int(bt.off[j + 1])
        n = b - a
        Z = _Z(Pm[a:b])
        u = qtw[3 * a:3 * b]
        wj = w[ro:ro + 3 * n - 6]
        ro += 3 * n - 6
        ann = max(ann, np.abs(Z @ u).max() / (np.abs(Z).max() * np.linalg.norm(wj)))
        iso = max(iso, abs(np.linalg.norm(u) - np.linalg.norm(wj)) / np.linalg.norm(wj))
        fj = f[3 * a:3 * b]
        Zc = _Z(Pm[a:b] - Pm[a:b].mean(0))  # same row space as Z, better conditioned
        want = fj - Zc.T @ np.linalg.solve(Zc @ Zc.T, Zc @ fj)
        proj = max(proj, np.linalg.norm(pf[3 * a:3 * b] - want) / np.linalg.norm(fj))
    return ann, iso, proj


def test_moved_body_complement(case):
    bt, Rm, Pm = case
    ann, iso, proj = _checks(bt, Rm, Pm, 5)
    assert ann < 1e-13 and iso < 1e-13 and proj < 1e-12, (ann, iso, proj)


def test_transposed_rotation_fails_the_pins(case):
    bt, Rm, Pm = case
    ann, _, proj = _checks(bt, np.transpose(Rm, (0, 2, 1)), Pm, 5)
    assert ann > 1e-3 and proj > 1e-3, (ann, proj)
