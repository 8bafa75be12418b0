"""Helpers of the GPU parity tests (test code only; no method arithmetic of
the library lives here).

compare_per_body holds every body's part of a product to the tolerance in
two ways at once: the relative 2-norm |got - ref| / |ref| of the body's
vector, and element by element, |got_i - ref_i| <= tol * s_i, so that one
wrong element cannot hide in a body's norm.  By default s_i = max_j |ref_j|
over the body.  For Q~v the element scale is the one rounding analysis
gives (residue_scales): the residues of node p are made by orthogonal
transforms from the bead vectors below p, so each is at most, and each
rounding error in it proportional to, the 2-norm of those bead vectors
(|v_sub(p)|; an error made below p travels up through orthogonal maps
without growth).  Near the root of a large body that norm is far above
the residues themselves (about 1.8e3 against residues of order 1 for the
2^20-bead body), so two correct FP64 implementations differ there by more
than 1e-12 of the body's largest residue; everywhere below, s_i is of the
order of the element itself.

record_to_G expands one exported FP64 node record (include/zq.h,
zq_get_records) into the dense k x k G it encodes, to compare it with the
oracle's G.
"""
from __future__ import annotations

import numpy as np


def body_slices(off, kind):
    """(start, stop) of every body in a residue vector (kind "res": 3n - 6
    entries per body) or an interleaved bead vector ("bead": 3n)."""
    out, ro = [], 0
    for j in range(len(off) - 1):
        o, n = int(off[j]), int(off[j + 1] - off[j])
        if kind == "res":
            out.append((ro, ro + 3 * n - 6))
        else:
            out.append((3 * o, 3 * (o + n)))
        ro += 3 * n - 6
    return out


def node_factors(B, x, y, z, tol, u):
    """Per node p of oracle body B: max(1, 8 cond(p) A(p) u / tol).

    cond(p) is the conditioning of the node's factorisation M = [T22 0] G
    (the singular values of M are those of T22): sigma_1 / sigma_3, or
    sigma_1 / sigma_2 for Case I nodes, whose T22 has rank two; 1 for
    singular (flagged) nodes, which both sides factorise through exact
    zeros.  A(p) = (|c_x| + |c_y|) / |c_x - c_y| is the cancellation in the
    offset d = c_x - c_y between the children's centroids: centroids are
    rounded sums of absolute coordinates (relative error u), so d, and with
    it M, is known only to about A(p) u relative, and G to cond(p) A(p) u
    (forward error of a backward-stable QR).  Two correct builds may differ
    by that much; u is the unit roundoff of the build's arithmetic."""
    L, C = B.nodes_all()
    t = B.tree()
    sv = np.linalg.svd(L, compute_uv=False)
    case1 = (t["left"] < 0) & (t["right"] < 0)
    den = np.where(case1, sv[:, 1], sv[:, 2])
    cond = np.where(den > 0, sv[:, 0] / np.where(den > 0, den, 1.0), 1.0)
    P = np.stack([x, y, z], 1)

    def cen(code):
        return np.where((code >= 0)[:, None], C[np.maximum(code, 0)], P[t["perm"][np.maximum(-1 - code, 0)]])

    cx, cy = cen(t["left"]), cen(t["right"])
    dn = np.linalg.norm(cx - cy, axis=1)
    A = np.where(dn > 0, (np.linalg.norm(cx, axis=1) + np.linalg.norm(cy, axis=1)) / np.where(dn > 0, dn, 1.0), 1.0)
    return np.maximum(1.0, 8.0 * cond * A * u / tol)


def _subtree_max(t, fac):
    """Max of fac over each node's subtree (the node included): an error
    made in a descendant's transform reaches the node's residues."""
    out = fac.copy()
    h = t["height"]
    for lev in range(2, int(h.max()) + 1):
        g = np.nonzero(h == lev)[0]
        for side in ("left", "right"):
            ch = t[side][g]
            inner = ch >= 0
            out[g[inner]] = np.maximum(out[g[inner]], out[ch[inner]])
    return out


def _ancestor_max_per_bead(t, fac, n):
    """Max of fac over each bead's ancestors, indexed by the body's bead
    index: the downward sweep carries every ancestor's transform error to
    the bead."""
    anc = fac.copy()
    bead = np.ones(n)
    h = t["height"]
    for lev in range(int(h.max()), 0, -1):
        g = np.nonzero(h == lev)[0]
        for side in ("left", "right"):
            ch = t[side][g]
            inner = ch >= 0
            anc[ch[inner]] = np.maximum(anc[ch[inner]], anc[g[inner]])
            leaf = ~inner
            bead[t["perm"][-1 - ch[leaf]]] = anc[g[leaf]]
    return bead


def residue_scales(off, x, y, z, f, tol=None, u=None):
    """For every residue of Q~v (the library's in-order layout), the 2-norm
    of the input bead vectors below the node that writes it, from the
    oracle's tree (f: interleaved bead vectors, 3N).

    With tol and u (the unit roundoff of the arithmetic the transforms were
    built in), each scale is multiplied by the largest node_factors value in
    the node's subtree, so that the element check holds each residue to
    max(tol, 8 cond A u) |v_sub(p)|."""
    import oracle

    out = []
    for j in range(len(off) - 1):
        o, n = int(off[j]), int(off[j + 1] - off[j])
        xs, ys, zs = x[o:o + n], y[o:o + n], z[o:o + n]
        B = oracle.Body(xs, ys, zs)
        t = B.tree()
        sq = (np.asarray(f[3 * o:3 * (o + n)]).reshape(n, 3) ** 2).sum(1)[t["perm"]]
        cs = np.concatenate([[0.0], np.cumsum(sq)])
        norm_p = np.sqrt(np.maximum(cs[t["last"] + 1] - cs[t["first"]], 0.0))
        if tol is not None and u is not None:
            norm_p = norm_p * _subtree_max(t, node_factors(B, xs, ys, zs, tol, u))
        nres = 3 * ((t["left"] >= 0).astype(np.int64) + (t["right"] >= 0).astype(np.int64))
        assert np.all(t["roff"] == np.concatenate([[0], np.cumsum(nres)[:-1]]))  # in-order offsets
        out.append(np.repeat(norm_p, nres))
    return np.concatenate(out)


def bead_scales(off, x, y, z, ref, tol, u):
    """For every element of Q~^T w (interleaved, 3N): the body's largest
    |ref| times the largest node_factors value among the bead's ancestors."""
    import oracle

    out = []
    for j in range(len(off) - 1):
        o, n = int(off[j]), int(off[j + 1] - off[j])
        xs, ys, zs = x[o:o + n], y[o:o + n], z[o:o + n]
        B = oracle.Body(xs, ys, zs)
        fb = _ancestor_max_per_bead(B.tree(), node_factors(B, xs, ys, zs, tol, u), n)
        out.append(np.repeat(fb, 3) * np.abs(ref[3 * o:3 * (o + n)]).max())
    return np.concatenate(out)


def errors_per_body(got, ref, off, kind, scale=None):
    """Per body: (relative 2-norm error, worst element error / its scale);
    scale None: the body's max |ref|."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    norm_err, elem_err = [], []
    for a, b in body_slices(off, kind):
        g, r = got[..., a:b], ref[..., a:b]
        if r.size == 0:
            norm_err.append(0.0)
            elem_err.append(0.0)
            continue
        d = np.abs(g - r)
        norm_err.append(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300))
        if not np.all(np.isfinite(g)):
            elem_err.append(np.inf)
        elif scale is None:
            elem_err.append(d.max() / max(np.abs(r).max(), 1e-300))
        else:
            elem_err.append((d / np.maximum(scale[a:b], 1e-300)).max())
    return np.array(norm_err), np.array(elem_err)


def compare_per_body(got, ref, off, kind, tol, what="", scale=None, elem_tol=None):
    """Asserts both per-body bounds (see the module docstring), the element
    bound at elem_tol if given (else tol); returns the worst (norm error,
    element error) for reporting."""
    ne, ee = errors_per_body(got, ref, off, kind, scale)
    jn, je = int(np.argmax(ne)), int(np.argmax(ee))
    et = tol if elem_tol is None else elem_tol
    assert ne[jn] <= tol, f"{what}: body {jn} relative 2-norm error {ne[jn]:.3e} > {tol:.1e}"
    assert ee[je] <= et, f"{what}: body {je} worst element error {ee[je]:.3e} x its scale > {et:.1e}"
    return float(ne[jn]), float(ee[je])


def compare_elementwise(got, ref, tol, what=""):
    """One vector (a single body): both bounds over the whole vector."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    ne = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
    ee = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    assert ne <= tol, f"{what}: relative 2-norm error {ne:.3e} > {tol:.1e}"
    assert ee <= tol, f"{what}: worst element error {ee:.3e} x max|ref| > {tol:.1e}"
    return float(ne), float(ee)


def record_to_G(rec: np.ndarray, k: int) -> np.ndarray:
    """Dense k x k G from one FP64 record: Case I stores G row-major in
    entries 5..13; otherwise G = D H_3 H_2 H_1 with H_j = I - |tau_j| v_j v_j^T
    (v_j(j) = 1, entries below it stored in order) and D_jj = -1 where the
    sign bit of tau_j is set."""
    if k == 3:
        return rec[5:14].reshape(3, 3).copy()
    G = np.eye(k)
    tail = 5
    for j in range(3):
        v = np.zeros(k)
        v[j] = 1.0
        v[j + 1:] = rec[tail:tail + k - 1 - j]
        tail += k - 1 - j
        G = G - abs(rec[2 + j]) * np.outer(v, v @ G)
    for j in range(3):
        if np.signbit(rec[2 + j]):
            G[j] = -G[j]
    return G
