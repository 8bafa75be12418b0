"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself:
the paper's printed closed form (Eqs. 3.9-3.10), LAPACK's Householder QR
(the paper factorises Eq. 3.5 with Matlab qr), the dense projector
I - Z^T (Z Z^T)^{-1} Z and an SVD complement of Z^T (Problem Statement,
Sec. 1), the rigid velocity field v_i = V + w x r_i (Sec. 4.2), an
independent real-arithmetic bisection (Sec. 2.1), and the magnitudes of
Table 1 (Sec. 5.2).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1708_08427_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def z_matrix(x, y, z):
    """Eq. 1.2: Z = [I ... I; A_1 ... A_n], A_k f = r_k x f."""
    n = x.shape[0]
    Z = np.zeros((6, 3 * n))
    for i in range(n):
        Z[0:3, 3 * i:3 * i + 3] = np.eye(3)
        Z[3:6, 3 * i:3 * i + 3] = [[0.0, -z[i], y[i]], [z[i], 0.0, -x[i]], [-y[i], x[i], 0.0]]
    return Z


def geometry(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "shell":
        b = W.shell_body(n, seed=seed)
        return b.x, b.y, b.z
    if kind == "cube":
        p = rng.uniform(-1, 1, (n, 3))
    elif kind == "far":      # body far from the origin (cancellation)
        p = rng.uniform(-1, 1, (n, 3)) + np.array([100.0, -70.0, 40.0])
    elif kind == "flat":     # beads on a plane z = const
        p = rng.uniform(-1, 1, (n, 3))
        p[:, 2] = 0.25
    elif kind == "clustered":
        p = np.concatenate([rng.normal(0, 1e-3, (n // 2, 3)), rng.normal(5, 1e-3, (n - n // 2, 3))])
    else:
        raise ValueError(kind)
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy()


# ---------------------------------------------------------------- Eq. 3.5


def qr_nonneg(A):
    """LAPACK's complete QR of A (k x 3) with the signs of R's diagonal made
    nonnegative (rows of R and columns of Q flipped together)."""
    Q, R = np.linalg.qr(A, mode="complete")
    sgn = np.ones(A.shape[0])
    sgn[:3] = np.where(np.diag(R[:3, :3]) < 0, -1.0, 1.0)
    return Q * sgn, sgn[:, None] * R


@pytest.mark.parametrize("k", [6, 9])
@pytest.mark.parametrize("seed", range(5))
def test_lq_matches_lapack_householder(k, seed):
    """Eq. 3.5 is computed with a Householder QR ('Matlab qr' = LAPACK
    dgeqrf/dorgqr; numpy's qr calls the same routines) whose R diagonal is
    then made nonnegative (T22 lower triangular with a nonnegative diagonal,
    the layout of Eq. 3.6).  For full-rank M that fixes T22 and G's first
    three rows uniquely; the completion rows are LAPACK's."""
    rng = np.random.default_rng(100 + seed)
    M = rng.standard_normal((3, k))
    if seed % 2:  # the structure of [R22 S22 K]: lower-triangular blocks and a skew block
        for b0 in range(0, k - 3, 3):
            M[:, b0:b0 + 3] = np.tril(M[:, b0:b0 + 3])
        d = rng.standard_normal(3)
        M[:, k - 3:] = [[0, -d[2], d[1]], [d[2], 0, -d[0]], [-d[1], d[0], 0]]
    L, G = oracle.lq(M)
    Q, R = qr_nonneg(M.T)
    np.testing.assert_allclose(L, R[:3, :3].T, atol=1e-14, rtol=0)
    np.testing.assert_allclose(G, Q.T, atol=1e-14, rtol=0)
    assert np.all(np.diag(L) >= 0.0)
    # and the defining properties
    np.testing.assert_allclose(G @ G.T, np.eye(k), atol=1e-14)
    np.testing.assert_allclose(np.hstack([L, np.zeros((3, k - 3))]) @ G, M, atol=1e-14)
    assert np.all(np.triu(L, 1) == 0.0)


# ---------------------------------------------------------- Eqs. 3.9-3.10


def _read_case_one():
    rows = []
    with open(os.path.join(GOLDEN, "case_one_eq3_9_3_10.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            abc, t22, u = line.split("|")
            rows.append((np.array(abc.split(), float), np.array(t22.split(), float).reshape(3, 3),
                         np.array(u.split(), float).reshape(3, 6)))
    return rows


def _case_one_node(a, b, c):
    """Beads at (a, b, c) (child x) and -(a, b, c) (child y): d = c_x - c_y,
    n_x = n_y = 1, sqrt(n_x n_y / n) = 1/sqrt(2); U = G C' with
    C' = [sqrt(n_y/n) I, -sqrt(n_x/n) I] (Theorem 3.2)."""
    L, G, dg = oracle.case_one(2.0 * np.array([a, b, c]), 1.0 / np.sqrt(2.0))
    U = np.hstack([G, -G]) / np.sqrt(2.0)
    return L, U, dg


@pytest.mark.parametrize("row", range(3))
def test_case_one_golden(row):
    abc, T22, U = _read_case_one()[row]
    L, Uo, dg = _case_one_node(*abc)
    assert not dg
    np.testing.assert_allclose(L, T22, atol=1e-14, rtol=0)
    np.testing.assert_allclose(Uo, U, atol=1e-14, rtol=0)


def test_case_one_printed_formula_random():
    """The printed Eqs. 3.9-3.10 at random (a, b, c) with b >= 0, c > 0."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        a = rng.normal()
        b = abs(rng.normal())
        c = abs(rng.normal()) + 1e-3
        s2 = b * b + c * c
        r2 = a * a + s2
        T22 = np.array([
            [np.sqrt(2 * s2), 0, 0],
            [-np.sqrt(2) * a * b / np.sqrt(s2), np.sqrt(2 * c * c * r2 / s2), 0],
            [-np.sqrt(2) * a * c / np.sqrt(s2), -np.sqrt(2 * b * b * r2 / s2), 0]])
        U = np.array([
            np.array([0, -c, b, 0, c, -b]) / np.sqrt(2 * s2),
            np.array([s2, -a * b, -a * c, -s2, a * b, a * c]) / np.sqrt(2 * r2 * s2),
            np.array([-a, -b, -c, a, b, c]) / np.sqrt(2 * r2)])
        L, Uo, _ = _case_one_node(a, b, c)
        np.testing.assert_allclose(L, T22, atol=1e-13)
        np.testing.assert_allclose(Uo, U, atol=1e-13)


def test_case_one_degenerate_and_axis():
    L, G, dg = oracle.case_one(np.zeros(3), 0.7)
    assert dg and np.all(L == 0) and np.all(G == np.eye(3))
    # d along x: still an orthogonal G with K = [L 0] G (rank two)
    d = np.array([1.5, 0.0, 0.0])
    L, G, dg = oracle.case_one(d, 0.7)
    K = 0.7 * np.array([[0, -d[2], d[1]], [d[2], 0, -d[0]], [-d[1], d[0], 0]])
    assert not dg
    np.testing.assert_allclose(G @ G.T, np.eye(3), atol=1e-15)
    np.testing.assert_allclose(L @ G, K, atol=1e-15)


# ------------------------------------------- Problem Statement, brute force


def projector(Z):
    """Orthogonal projector onto the row space of Z, from a QR of Z^T (stable
    even when Z Z^T is ill-conditioned, e.g. two tight far-apart clusters)."""
    Q, _ = np.linalg.qr(Z.T)
    return Q @ Q.T


def _svd_complement(Z):
    """Orthonormal basis of the orthogonal complement of the row space of Z."""
    U, s, _ = np.linalg.svd(Z.T, full_matrices=True)
    r = int(np.sum(s > 1e-10 * s[0]))
    return U[:, r:].T


@pytest.mark.parametrize("kind", ["shell", "cube", "far", "flat", "clustered"])
@pytest.mark.parametrize("n", [3, 4, 5, 8, 17, 40, 64])
def test_dense_complement_brute_force(kind, n):
    x, y, z = geometry(kind, n, seed=n)
    B = oracle.Body(x, y, z)
    Qt, QZ = B.qgen()
    Z = z_matrix(x, y, z)
    n3 = 3 * n
    assert Qt.shape == (n3 - 6, n3)
    np.testing.assert_allclose(Qt @ Qt.T, np.eye(n3 - 6), atol=1e-13)
    assert np.abs(Qt @ Z.T).max() <= 1e-12 * max(1.0, np.abs(Z).max())
    P = projector(Z)
    np.testing.assert_allclose(Qt.T @ Qt, np.eye(n3) - P, atol=1e-11)
    C = _svd_complement(Z)
    np.testing.assert_allclose(Qt.T @ Qt, C.T @ C, atol=1e-11)
    # Q = [Q_Z; Q~] is orthogonal and Q_Z spans the rows of Z (Eq. 3.3)
    Q = np.vstack([QZ, Qt])
    np.testing.assert_allclose(Q @ Q.T, np.eye(n3), atol=1e-13)
    coef = np.linalg.lstsq(QZ.T, Z.T, rcond=None)[0]
    np.testing.assert_allclose(QZ.T @ coef, Z.T, atol=1e-10 * max(1.0, np.abs(Z).max()))


@pytest.mark.parametrize("kind", ["shell", "cube", "flat"])
@pytest.mark.parametrize("n", [5, 33, 64])
def test_implicit_passes_match_projector(kind, n):
    """Q~^T Q~ v = v - Z^T (Z Z^T)^{-1} Z v and ||Q~^T w|| = ||w||."""
    x, y, z = geometry(kind, n, seed=3 * n)
    B = oracle.Body(x, y, z)
    Z = z_matrix(x, y, z)
    rng = np.random.default_rng(n)
    for _ in range(4):
        v = rng.standard_normal(3 * n)
        proj = v - projector(Z) @ v
        np.testing.assert_allclose(B.apply_QT(B.apply_Q(v)), proj, atol=1e-11)
        w = rng.standard_normal(3 * n - 6)
        qtw = B.apply_QT(w)
        assert abs(np.linalg.norm(qtw) - np.linalg.norm(w)) <= 1e-12 * np.linalg.norm(w)
        np.testing.assert_allclose(Z @ qtw, 0.0, atol=1e-11 * max(1.0, np.abs(Z).max()))


def test_single_body_basic_shapes():
    x, y, z = geometry("cube", 3, seed=1)
    B = oracle.Body(x, y, z)
    t = B.tree()
    # n = 3: one Case I node and one Case II node; residue dimension 3 = 3n - 6
    ks = sorted(B.node(g)["k"] for g in range(2))
    assert ks == [3, 6]
    assert t["roff"].tolist() in ([0, 0], [0, 3])


# ------------------------------------------- O(n) invariants at larger n


@pytest.mark.parametrize("n", [1000, 20000])
def test_invariants_large(n):
    b = W.shell_body(n, radius=0.1 * np.sqrt(n), sigma=0.0025 * np.sqrt(n), seed=5,
                     centre=(60.0, 20.0, 80.0))
    B = oracle.Body(b.x, b.y, b.z)
    rng = np.random.default_rng(11)
    r = np.stack([b.x, b.y, b.z], 1)
    # rigid field v_i = V + omega x r_i (Sec. 4.2) is annihilated by Q~
    V, om = rng.standard_normal(3), rng.standard_normal(3)
    v_rigid = (V + np.cross(om, r)).reshape(-1)
    assert np.linalg.norm(B.apply_Q(v_rigid)) <= 1e-12 * np.linalg.norm(v_rigid)
    # Parseval: ||Q~ v||^2 + ||Q_Z v||^2 = ||v||^2, and Q_Z v = root Info-set
    v = rng.standard_normal(3 * n)
    qv, root = B.apply_Q(v, with_root=True)
    assert abs(qv @ qv + root @ root - v @ v) <= 1e-11 * (v @ v)
    # the root translational Info-set is sum(f)/sqrt(n) (Definition 4.1)
    np.testing.assert_allclose(root[:3], v.reshape(-1, 3).sum(0) / np.sqrt(n), atol=1e-11)
    # Q~^T w carries no net force and no net torque (Z Q~^T = 0)
    w = rng.standard_normal(3 * n - 6)
    out = B.apply_QT(w).reshape(-1, 3)
    scale = np.linalg.norm(w) * np.abs(r).max()
    assert np.abs(out.sum(0)).max() <= 1e-12 * scale
    assert np.abs(np.cross(r, out).sum(0)).max() <= 1e-11 * scale


# ------------------------------------------------------- Table 1, Sec. 5.2


def _table1():
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_orthogonality.txt"))
    return rows[:, 1:].max(axis=0)


@pytest.mark.parametrize("n", [500, 1000])
def test_table1_orthogonality(n):
    """The oracle reproduces the six Table 1 measures at or below the worst
    value the paper reports for any n."""
    bound = _table1()
    b = W.shell_body(n, radius=0.1 * np.sqrt(n), sigma=0.0025 * np.sqrt(n), seed=n)
    B = oracle.Body(b.x, b.y, b.z)
    Qt, QZ = B.qgen()
    Q = np.vstack([QZ, Qt])
    n3 = 3 * n
    rng = np.random.default_rng(n)
    v = rng.standard_normal(n3)
    qv, root = B.apply_Q(v, with_root=True)
    errs = [
        np.abs(Q @ Q.T - np.eye(n3)).max(),
        np.abs(Q.T @ Q - np.eye(n3)).max(),
        np.abs(np.concatenate([root, qv]) - Q @ v).max(),
        np.abs(B.apply_QT(v[6:], v[:6]) - Q.T @ v).max(),
        np.abs(B.apply_QT(qv, root) - v).max(),
    ]
    Qtv = B.apply_QT(v[6:], v[:6])
    q2, r2 = B.apply_Q(Qtv, with_root=True)
    errs.append(np.abs(np.concatenate([r2, q2]) - v).max())
    for e, bd in zip(errs, bound):
        assert e <= bd, (errs, bound)


# ------------------------------------------------------------- Sec. 2.1


def _bisect_real(x, y, z):
    """The tree of Sec. 2.1 built directly from real coordinates: the root box
    is normalised to side 1; each box is split at its midpoint along z, then
    y, then x; empty boxes are pruned; a box with one bead is a leaf.
    Returns (perm, {g: (left, right, first, last)})."""
    n = x.shape[0]
    P = np.stack([x, y, z], 1)
    lo, hi = P.min(0), P.max(0)
    T = np.where(hi > lo, (P - lo) / np.where(hi > lo, hi - lo, 1.0), 0.0)
    perm, nodes = [], {}

    def rec(S, box_lo, box_hi, level, pos):
        if len(S) == 1:
            perm.append(S[0])
            return -1 - pos
        while True:
            axis = 2 - level % 3
            mid = 0.5 * (box_lo[axis] + box_hi[axis])
            up = [i for i in S if T[i, axis] >= mid]
            dn = [i for i in S if T[i, axis] < mid]
            lo2, hi2 = box_lo.copy(), box_hi.copy()
            hi2[axis] = mid
            lo3, hi3 = box_lo.copy(), box_hi.copy()
            lo3[axis] = mid
            level += 1
            if dn and up:
                break
            if dn:
                box_lo, box_hi = lo2, hi2
            else:
                box_lo, box_hi = lo3, hi3
            assert level < 63, "beads closer than the 21-bit resolution"
        lc = rec(dn, lo2, hi2, level, pos)
        rc = rec(up, lo3, hi3, level, pos + len(dn))
        g = pos + len(dn) - 1
        nodes[g] = (lc, rc, pos, pos + len(S) - 1)
        return g

    rec(list(range(n)), np.zeros(3), np.ones(3), 0, 0)
    return np.array(perm), nodes


@pytest.mark.parametrize("kind", ["shell", "cube", "far", "flat"])
@pytest.mark.parametrize("n", [3, 9, 50, 300])
def test_tree_matches_real_bisection(kind, n):
    x, y, z = geometry(kind, n, seed=n + 1)
    t = oracle.Body(x, y, z).tree()
    perm, nodes = _bisect_real(x, y, z)
    np.testing.assert_array_equal(t["perm"], perm)
    for g, (lc, rc, f, l) in nodes.items():
        assert (t["left"][g], t["right"][g], t["first"][g], t["last"][g]) == (lc, rc, f, l)


def test_tree_ties_split_by_index():
    """Coincident beads (same 21-bit cell) are separated by their index bits."""
    x = np.array([0.0, 1.0, 0.5, 0.5, 0.5])
    y = np.array([0.0, 1.0, 0.5, 0.5, 0.5])
    z = np.array([0.0, 1.0, 0.5, 0.5, 0.5])
    t = oracle.Body(x, y, z).tree()
    # beads 2, 3, 4 share a cell; index order 2 < 3 < 4 is kept
    pos = {b: i for i, b in enumerate(t["perm"])}
    assert pos[2] < pos[3] < pos[4]
    assert t["roff"][-1] + 3 * int(t["left"][-1] >= 0) + 3 * int(t["right"][-1] >= 0) == 3 * 5 - 6


@pytest.mark.parametrize("n", [3, 10, 100, 1000])
def test_residue_dimensions(n):
    x, y, z = geometry("cube", n, seed=2)
    B = oracle.Body(x, y, z)
    t = B.tree()
    sizes = [B.node(g)["k"] - 3 for g in range(n - 1)]
    assert sum(sizes) == 3 * n - 6
    for g in range(n - 1):
        internal = int(t["left"][g] >= 0) + int(t["right"][g] >= 0)
        assert sizes[g] == 3 * internal
    np.testing.assert_array_equal(t["roff"], np.concatenate([[0], np.cumsum(sizes)[:-1]]))


def test_translation_invariance():
    x, y, z = geometry("cube", 50, seed=9)
    B0 = oracle.Body(x, y, z)
    B1 = oracle.Body(x + 3.0, y - 1.0, z + 0.5)
    Q0, _ = B0.qgen()
    Q1, _ = B1.qgen()
    np.testing.assert_allclose(Q0, Q1, atol=1e-12)


def test_batch_is_block_diagonal():
    """Sec. 1: Q~ = diag(Q~^1, ..., Q~^m)."""
    bt = W.shell_batch(m=5, nmin=5, nmax=40, seed=3)
    rng = np.random.default_rng(0)
    f = rng.standard_normal(3 * bt.N)
    w = rng.standard_normal(bt.n_residues)
    qf, qtw = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, f, w)
    ro = 0
    for j in range(bt.m):
        a, b = bt.off[j], bt.off[j + 1]
        B = oracle.Body(*bt.body(j))
        n = b - a
        np.testing.assert_array_equal(qf[ro:ro + 3 * n - 6], B.apply_Q(f[3 * a:3 * b]))
        np.testing.assert_array_equal(qtw[3 * a:3 * b], B.apply_QT(w[ro:ro + 3 * n - 6]))
        ro += 3 * n - 6


# ------------------------------------------- node assembly, Eq. 3.5 as printed


def _cross(a):
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def _pair_T22(ra, rb):
    """T22 of a bead pair (child x = ra, child y = rb) from Eq. 3.10: the rows
    of U are g_i [1, -1]/sqrt(2); T22 follows from Eq. 3.5 as K G^T with
    K = sqrt(n_x n / n_y) R21 = sqrt(2) [ra - c]x, c the pair's centroid."""
    c = 0.5 * (ra + rb)
    a, b, cc = ra - c
    s2, r2 = b * b + cc * cc, a * a + b * b + cc * cc
    G = np.array([np.array([0, -cc, b]) / np.sqrt(s2),
                  np.array([s2, -a * b, -a * cc]) / np.sqrt(r2 * s2),
                  np.array([-a, -b, -cc]) / np.sqrt(r2)])
    K = np.sqrt(2.0) * _cross(ra - c)
    T22 = K @ G.T
    T22[:, 2] = 0.0   # Eq. 3.9: the third column is exactly zero (rank two)
    return T22, c


@pytest.mark.parametrize("seed", range(6))
def test_node_assembly_eq_3_5(seed):
    """Root of a 4-bead body whose children are two bead pairs: the oracle's
    T22 and G equal the LQ (LAPACK) of [R22 S22 sqrt(n_x n/n_y) R21] built
    term by term from Eq. 3.5 with R21 = [c_x - c_p]x; and for a 3-bead body
    (Case II, Eqs. 3.11-3.13) the 3 x 6 form with the single bead's block
    dropped."""
    rng = np.random.default_rng(200 + seed)
    # two well separated pairs: the first bisection (z) separates the pairs
    p = np.array([[0.1, 0.2, 0.1], [0.9, 0.7, 0.3], [0.2, 0.8, 2.6], [0.8, 0.1, 2.9]])
    p += rng.normal(0, 0.03, p.shape)
    B = oracle.Body(p[:, 0], p[:, 1], p[:, 2])
    t = B.tree()
    root = t["root"]
    lx, ly = t["left"][root], t["right"][root]
    assert lx >= 0 and ly >= 0
    pair = lambda g: [p[t["perm"][t["first"][g]]], p[t["perm"][t["last"][g]]]]
    R22, cx = _pair_T22(*pair(lx))
    S22, cy = _pair_T22(*pair(ly))
    cp = 0.25 * p.sum(0)
    M = np.hstack([R22, S22, np.sqrt(2 * 4 / 2) * _cross(cx - cp)])
    Q, R = qr_nonneg(M.T)
    nd = B.node(root)
    np.testing.assert_allclose(nd["L"], R[:3, :3].T, atol=1e-13)
    np.testing.assert_allclose(nd["G"], Q.T, atol=1e-13)
    np.testing.assert_allclose(nd["c"], cp, atol=1e-15)
    # Case II: drop the last bead; the pair and the single bead meet at the root
    p3 = p[:3]
    B3 = oracle.Body(p3[:, 0], p3[:, 1], p3[:, 2])
    t3 = B3.tree()
    r3 = t3["root"]
    lx, ly = t3["left"][r3], t3["right"][r3]
    cp = p3.mean(0)
    if lx >= 0:   # x = the pair, y = the bead (Eqs. 3.11-3.13 as printed)
        R22, cx = _pair_T22(*pair_of(t3, p3, lx))
        M = np.hstack([R22, np.sqrt(2 * 3 / 1) * _cross(cx - cp)])
    else:         # x = the bead, y = the pair
        S22, _ = _pair_T22(*pair_of(t3, p3, ly))
        cx = p3[t3["perm"][t3["first"][r3]]]
        M = np.hstack([S22, np.sqrt(1 * 3 / 2) * _cross(cx - cp)])
    Q, R = qr_nonneg(M.T)
    nd = B3.node(r3)
    np.testing.assert_allclose(nd["L"], R[:3, :3].T, atol=1e-13)
    np.testing.assert_allclose(nd["G"], Q.T, atol=1e-13)


def pair_of(t, p, g):
    return [p[t["perm"][t["first"][g]]], p[t["perm"][t["last"][g]]]]


# ----------------------------------------------- rank-deficient nodes (A8)


def test_lq_rank_deficient_is_exact_and_valid():
    """M = [0 | K] (a child whose beads coincide, T22 = 0, next to a bead):
    rank two.  The third pivot is exactly zero, L G = M, G orthogonal, and
    the completion rows annihilate M's rows."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        d = rng.standard_normal(3)
        K = 0.8 * _cross(d)
        for M in (np.hstack([np.zeros((3, 3)), K]), np.hstack([np.zeros((3, 3)), np.zeros((3, 3)), K])):
            k = M.shape[1]
            L, G = oracle.lq(M)
            assert L[2, 2] == 0.0
            np.testing.assert_allclose(G @ G.T, np.eye(k), atol=1e-14)
            np.testing.assert_allclose(np.hstack([L, np.zeros((3, k - 3))]) @ G, M, atol=1e-14)
            np.testing.assert_allclose(M @ G[3:].T, 0.0, atol=1e-14)


def _scaled_full_rank_M(rng, k, e):
    """M = [s T22_x | (T22_y) | K] with the child block s T22_x lower
    triangular, entries of magnitude [1/2, 1) s, s = 2^-e, beside an O(1)
    skew block K = [d]x (rank two) and, for k = 9, an O(1) lower-triangular
    T22_y: a full-rank M whose third singular value is about s |M| (a tight
    child cluster next to a far sibling)."""
    sgn = lambda shape: rng.choice([-1.0, 1.0], shape)
    d = rng.uniform(0.5, 1.0, 3) * sgn(3)
    T = np.tril(rng.uniform(0.5, 1.0, (3, 3)) * sgn((3, 3))) * 2.0 ** -e
    if k == 6:
        return np.hstack([T, _cross(d)])
    T2 = np.tril(rng.uniform(0.5, 1.0, (3, 3)) * sgn((3, 3)))
    return np.hstack([T, T2, _cross(d)])


@pytest.mark.parametrize("e", [10, 20, 30, 33, 36, 38, 39, 40])
def test_lq_badly_scaled_full_rank_matches_lapack(e):
    """Full-rank M whose child block is 2^-e of the rest (e <= 40): the
    numerical rank decision must not fire, so the oracle's G equals LAPACK's
    Householder QR (Matlab qr) of M^T up to the forward error of a
    backward-stable QR, 8 cond(M) 2^-53, and T22 likewise.  A rule that
    zeroed small entries one by one (rather than whole noise columns)
    perturbs the third pivot column by up to 2^-40 |M| against a column
    norm of about 2^-e |M| and fails this bound by orders of magnitude."""
    rng = np.random.default_rng(500 + e)
    u = 2.0 ** -53
    for _ in range(60):
        for k in (6, 9):
            M = _scaled_full_rank_M(rng, k, e)
            L, G = oracle.lq(M)
            Q, R = qr_nonneg(M.T)
            kap = np.linalg.cond(M)
            assert np.abs(G - Q.T).max() <= 8.0 * kap * u, (k, e, np.abs(G - Q.T).max() / (kap * u))
            assert np.abs(L - R[:3, :3].T).max() <= 8.0 * kap * u * np.abs(M).max()
            assert np.all(np.diag(L) > 0.0)


@pytest.mark.parametrize("e", [41, 42, 45, 50, 60])
def test_lq_below_rank_threshold_is_a_small_backward_perturbation(e):
    """Below the threshold (child block 2^-e of |M|, e > 40) the third
    column is rounding-level relative to M: the oracle treats M as rank two,
    and its factorisation is then the exact LQ of a matrix within
    2^-40 sqrt(k) max|M| of M: G orthogonal, [T22 0] G = M to that bound,
    T22 lower triangular with a nonnegative diagonal."""
    rng = np.random.default_rng(600 + e)
    for _ in range(60):
        for k in (6, 9):
            M = _scaled_full_rank_M(rng, k, e)
            L, G = oracle.lq(M)
            np.testing.assert_allclose(G @ G.T, np.eye(k), atol=1e-14)
            back = np.abs(np.hstack([L, np.zeros((3, k - 3))]) @ G - M).max()
            assert back <= 2.0 ** -40 * np.sqrt(k) * np.abs(M).max(), (k, e, back)
            assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) >= 0.0)


@pytest.mark.parametrize("n", [6, 13, 30])
def test_collinear_and_lattice_bodies(n):
    """Exactly collinear beads (rank Z = 5) and a lattice (many collinear
    triples): rows orthonormal and orthogonal to Z."""
    line = np.c_[np.arange(n) * 0.25, np.arange(n) * 0.5, np.full(n, 1.0)]
    g = np.arange(n)
    lattice = np.c_[g % 3, (g // 3) % 3, g // 9].astype(float)
    for p in (line, lattice):
        B = oracle.Body(p[:, 0], p[:, 1], p[:, 2])
        Qt, _ = B.qgen()
        Z = z_matrix(p[:, 0], p[:, 1], p[:, 2])
        np.testing.assert_allclose(Qt @ Qt.T, np.eye(3 * n - 6), atol=1e-13)
        assert np.abs(Qt @ Z.T).max() <= 1e-12 * np.abs(Z).max()


def _collinear_int(P):
    """Exact collinearity of integer points (all cross products zero)."""
    d = P[1:] - P[0]
    nz = d[np.any(d != 0, axis=1)]
    if len(nz) == 0:
        return True
    return bool(np.all(np.cross(nz[0], nz) == 0))


@pytest.mark.parametrize("n", [12, 27, 40])
def test_singular_T22_flag_marks_exactly_the_collinear_nodes(n):
    """A node's T22 is singular exactly when its beads are collinear (the
    centred rotational rows of Z_p then have rank two, Eq. 3.3); on integer
    lattices collinearity is decided exactly, so the flag must match it on
    every node, and no node of a jittered shell is flagged."""
    g = np.arange(n)
    for P in (np.c_[g % 3, (g // 3) % 3, g // 9], np.c_[g, 2 * g, np.full(n, 5)],
              np.c_[g % 4, g // 4, (g * 7) % 5]):
        P = P.astype(np.int64)
        B = oracle.Body(*(P[:, a].astype(float) for a in range(3)))
        t = B.tree()
        for q in range(n - 1):
            nd = B.node(q)
            beads = t["perm"][t["first"][q]:t["last"][q] + 1]
            if nd["k"] == 3:
                assert not nd["degenerate"]  # distinct beads
            else:
                assert nd["degenerate"] == _collinear_int(P[beads]), (q, P[beads])
    bt = W.shell_body(n=300, seed=5)
    B = oracle.Body(bt.x, bt.y, bt.z)
    assert not any(B.node(q)["degenerate"] for q in range(299))
