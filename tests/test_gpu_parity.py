"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tree and index construction: bit-exact.  FP64 transforms and sweeps:
relative error <= 1e-12; FP32 sweeps: <= 1e-5, per body, both as the
2-norm relative to the oracle's result and element by element: every
residue of Q~v within tol * the norm of the bead vectors below its node
(the scale of its rounding error), every element of Q~^T w within tol *
the body's largest |element|, each widened where the geometry itself
limits what any FP64 build can agree on: to 8 cond A u for nodes whose
factorisation has condition number cond, offset cancellation A = (|c_x| +
|c_y|) / |c_x - c_y|, and build roundoff u (2^-53 FP64, 2^-48
double-single), over the node's subtree (Q~v) or the bead's ancestors
(Q~^T w); tests/_parity.py. Sizes span many thread
blocks, per-height launches and per-body launches, with ragged bucket
boundaries; edge cases: 3-bead bodies, flat and far-off bodies, coincident
beads, collinear and lattice bodies, bodies that need the device radix sort,
the lowest and highest level cut, and the full-size workloads.
"""
import numpy as np
import pytest

import oracle
from _parity import bead_scales, compare_per_body, record_to_G, residue_scales
from paper_1708_08427_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {np.float64: 1e-12, np.float32: 1e-5}
# unit roundoff of the transform build: native FP64, or double-single (a
# 48-bit significand)
BUILD_U = {"fp64": 2.0 ** -53, "dd": 2.0 ** -48}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _zq():
    from paper_1708_08427_gb300 import zq

    return zq


def make_ctx(bt, cut=0, arith="dd"):
    dev = _dev()
    zq = _zq()
    x, y, z = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(0)
    ctx.set_build_arith(arith)
    ctx.build_tree_batched(bt.off, x, y, z, cut)
    ctx.build_transforms(x, y, z)
    ctx.test_arith = arith
    return ctx, (x, y, z)


def oracle_bodies(bt):
    return [oracle.Body(*bt.body(j)) for j in range(bt.m)]


def oracle_tree_global(bt, bodies):
    """The oracle's per-body trees in the library's global numbering."""
    N, m = bt.N, bt.m
    perm = np.empty(N, np.int32)
    nodes = N - m
    out = {k: np.empty(nodes, np.int64) for k in ("left", "right", "first", "count", "height", "roff")}
    rbase = 0
    for j, B in enumerate(bodies):
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        nb = o - j
        t = B.tree()
        perm[o:o + n] = t["perm"] + o
        sl = slice(nb, nb + n - 1)

        def glob(code):
            return np.where(code >= 0, code + nb, -1 - (o + (-1 - code)))

        out["left"][sl] = glob(t["left"])
        out["right"][sl] = glob(t["right"])
        out["first"][sl] = t["first"] + o
        out["count"][sl] = t["last"] - t["first"] + 1
        out["height"][sl] = t["height"]
        out["roff"][sl] = t["roff"] + rbase
        rbase += 3 * n - 6
    return perm, out


def check_tree(ctx, bt, bodies):
    g = ctx.get_tree()
    perm, ref = oracle_tree_global(bt, bodies)
    np.testing.assert_array_equal(g["perm"], perm)
    for k in ("left", "right", "first", "count", "height", "roff"):
        np.testing.assert_array_equal(g[k], ref[k], err_msg=k)


def check_nodes(ctx, bt, bodies):
    c, L = ctx.get_nodes()
    worst = 0.0
    for j, B in enumerate(bodies):
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        nb = o - j
        for gsp in range(n - 1):
            nd = B.node(gsp)
            Lo = nd["L"][np.tril_indices(3)]
            scale = max(np.abs(Lo).max(), 1e-300)
            worst = max(worst, np.abs(L[nb + gsp] - Lo).max() / scale)
            cs = max(np.abs(nd["c"]).max(), 1.0)
            worst = max(worst, np.abs(c[nb + gsp] - nd["c"]).max() / cs)
    assert worst <= 1e-12, worst
    return worst


def check_records(ctx, bt, bodies, arith, skip=()):
    """The exported FP64 transforms (Householder records with the sign bits
    of tau carrying T22's diagonal normalisation, or Case I's explicit G)
    expand to the oracle's G node by node.  G's sensitivity to a
    perturbation of M grows with the condition number of T22 (QR
    perturbation bound |dG| <~ cond(T22) * |dM| / |M|), so each node is held
    to max(1e-12, 8 * cond(T22) * u), u the relative perturbation: 2^-53 for
    the FP64 build; for the double-single build 2^-48 plus 2^-40, because
    its rounded entries can fall on the other side of a binade boundary
    than the oracle's, so that the numerical-zero rule (entries more than 40
    binary orders below max |M| set to zero) drops an entry of size about
    2^-40 |M| on one side only.  Flagged (singular) nodes go through exact
    zeros and are held to 1e-12.  Bodies listed in `skip` sit far from the
    origin: there G depends on differences of FP64 centroids of size |c|,
    whose last-bit rounding (|c| 2^-53 each, different in the oracle's and
    the kernel's order of operations) is not a property of the method;
    their products are checked by the sweeps."""
    u = 2.0 ** -48 + 2.0 ** -40 if arith == "dd" else 2.0 ** -53
    rec = ctx.get_records()
    worst = 0.0
    for j, B in enumerate(bodies):
        if j in skip:
            continue
        o, n = int(bt.off[j]), int(bt.off[j + 1] - bt.off[j])
        nb = o - j
        for gsp in range(n - 1):
            nd = B.node(gsp)
            G = record_to_G(rec[nb + gsp], nd["k"])
            cond = np.linalg.cond(nd["L"]) if nd["k"] > 3 and not nd["degenerate"] else 0.0
            tol = max(1e-12, 8.0 * cond * u)
            r = np.abs(G - nd["G"]).max() / tol
            assert r <= 1.0, (j, gsp, nd["k"], cond, r * tol)
            worst = max(worst, r)
    return worst


def check_apply(ctx, bt, dtype, k=1, seed=0, tol=None):
    """Q~v and Q~^T w of k random vectors against the oracle, every body held
    to the tolerance by its 2-norm and element by element; returns the worst
    (norm, element) errors."""
    dev = _dev()
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((k, 3, bt.N))
    w = rng.standard_normal((k, bt.n_residues))
    qv = ctx.apply_Q(torch.from_numpy(v).to(dev, getattr(torch, np.dtype(dtype).name)))
    qtw = ctx.apply_QT(torch.from_numpy(w).to(dev, getattr(torch, np.dtype(dtype).name)))
    ctx.sync(allow_degenerate=True)
    qv = qv.double().cpu().numpy()
    qtw = qtw.double().cpu().numpy()
    tol = tol or TOL[dtype]
    u = BUILD_U[getattr(ctx, "test_arith", "dd")]
    worst = (0.0, 0.0)
    for c in range(k):
        f = W.interleave(*v[c])
        rq, rqt = oracle.batch_apply(bt.off, bt.x, bt.y, bt.z, f, w[c])
        e1 = compare_per_body(qv[c], rq, bt.off, "res", tol, f"Q~v {np.dtype(dtype).name} column {c}",
                              scale=residue_scales(bt.off, bt.x, bt.y, bt.z, f, tol, u))
        e2 = compare_per_body(W.interleave(*qtw[c]), rqt, bt.off, "bead", tol,
                              f"Q~^T w {np.dtype(dtype).name} column {c}",
                              scale=bead_scales(bt.off, bt.x, bt.y, bt.z, rqt, tol, u))
        worst = tuple(max(a, b, d) for a, b, d in zip(worst, e1, e2))
    return worst


# --------------------------------------------------------------- cases


@pytest.mark.parametrize("arith", ["dd", "fp64"])
def test_single_body_256_sixteen_vectors(arith):
    """n = 256 shell of radius 2 with N(0, 0.05^2) jitter, 16 right-hand
    sides; bisection tree exact, FP64 and FP32 sweeps, transforms built in
    double-single and in native FP64."""
    bt = W.shell_body(256, radius=2.0, sigma=0.05, seed=0)
    ctx, _ = make_ctx(bt, cut=3, arith=arith)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    check_nodes(ctx, bt, bodies)
    check_records(ctx, bt, bodies, arith)
    check_apply(ctx, bt, np.float64, k=16, seed=1)
    check_apply(ctx, bt, np.float32, k=16, seed=1)


@pytest.mark.parametrize("cut,arith", [(1, "dd"), (4, "fp64"), (15, "dd"), (21, "fp64")])
def test_batch_ragged_levels(cut, arith):
    """Bodies from 3 to 700 beads; a low level cut sends most nodes through
    the per-body kernels, a high one through the per-height kernels; bucket
    boundaries fall inside warps; 3-bead bodies."""
    bt = W.shell_batch(m=60, nmin=3, nmax=700, seed=4)
    ctx, _ = make_ctx(bt, cut=cut, arith=arith)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    check_nodes(ctx, bt, bodies)
    check_apply(ctx, bt, np.float64, seed=2)
    check_apply(ctx, bt, np.float32, seed=3)


def test_results_do_not_depend_on_level_cut():
    """Every level cut the tuner can pick (and the extremes 1 and 6) gives
    the same bits for both products in both precisions."""
    from paper_1708_08427_gb300.tune import CUTS

    bt = W.shell_batch(m=60, nmin=50, nmax=5000, seed=8)
    dev = _dev()
    rng = np.random.default_rng(5)
    v = torch.from_numpy(rng.standard_normal((3, bt.N))).to(dev)
    w = torch.from_numpy(rng.standard_normal(bt.n_residues)).to(dev)
    outs = []
    for cut in sorted({1, 6, *CUTS}):
        ctx, _ = make_ctx(bt, cut=cut)
        outs.append((ctx.apply_Q(v).cpu(), ctx.apply_QT(w).cpu(),
                     ctx.apply_Q(v.float()).cpu(), ctx.apply_QT(w.float()).cpu()))
        ctx.sync()
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)


def test_size_class_and_segment_boundaries():
    """Bodies on both sides of every size boundary of the schedules: the
    per-block tree classes (1024, 2048, 4096, 8192 beads; 8193 goes to the
    device-wide sort), the 512-bead segments (a whole-body segment, and a
    body with one node above its segments) and the 64-top-node warp path:
    tree bit-exact, both products against the oracle."""
    sizes = [511, 512, 513, 1024, 1025, 2048, 2049, 4096, 4097, 8192, 8193]
    bodies = [np.stack(W.shell_body(n, seed=70 + i).body(0), 1) for i, n in enumerate(sizes)]
    bt = _batch_from_points(bodies)
    ctx, _ = make_ctx(bt, cut=12)
    ob = oracle_bodies(bt)
    check_tree(ctx, bt, ob)
    check_apply(ctx, bt, np.float64, seed=11)
    check_apply(ctx, bt, np.float32, seed=11)


def test_large_body_runs_of_shared_high_bits():
    """A body above the per-block sort limit whose beads share their high 32
    key bits in runs of every kind the device sort handles after its four
    high passes: pairs and short runs (insertion fix-up), a run of 40 and a
    run of 1500 beads spread over a few finest cells (one thread block,
    LSD passes over the low key bits, the longer one over two tiles), and a
    run of 300 beads in one finest cell (equal keys: index order).  The tree
    is bit-exact with the oracle's; the products are held to the
    conditioning of the clusters (as in test_tight_clusters_sort_exactly)."""
    rng = np.random.default_rng(77)
    spread = rng.uniform(-3, 3, (9000, 3))
    pairs = np.repeat(rng.uniform(-3, 3, (20, 3)), 2, axis=0) + 1e-8 * rng.uniform(0, 1, (40, 3))
    pts = np.r_[spread, pairs,
                0.5 + 1e-5 * rng.uniform(0, 1, (40, 3)),
                -1.0 + 1e-5 * rng.uniform(0, 1, (1500, 3)),
                2.0 + 1e-9 * rng.uniform(0, 1, (300, 3))]
    pts = pts[rng.permutation(len(pts))]
    bt = _batch_from_points([pts])
    assert bt.N > 8192
    ctx, _ = make_ctx(bt, cut=8)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    tol = max(TOL[np.float64], 8 * 2 * 3.0 * 2.0 ** -53 / 1e-9)
    check_apply(ctx, bt, np.float64, tol=tol)


def test_large_body_radix_sort_path():
    """A body above the per-block sort limit (device radix sort), with many
    nodes above the level cut (one block for the whole body's top)."""
    bt = W.ellipsoid_body(n=20000, seed=3)
    ctx, _ = make_ctx(bt, cut=8)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    check_nodes(ctx, bt, bodies)
    check_apply(ctx, bt, np.float64)
    check_apply(ctx, bt, np.float32)


def _boundary_body(rng, n, lo, size):
    """n beads of a body with bounding box [lo, lo + size]^3 (corners
    included), most of them on, or one ulp either side of, the boundaries
    of the 2^21 quantisation cells of each axis (the beads whose keys the
    tree kernels decide by the exact formula), the rest uniform."""
    hi = lo + size
    w = (hi - lo) / 2.0 ** 21
    cells = rng.integers(0, 2 ** 21, (n, 3))
    P = lo + cells * w
    step = rng.integers(-1, 2, (n, 3))
    P = np.where(step > 0, np.nextafter(P, np.inf), np.where(step < 0, np.nextafter(P, -np.inf), P))
    uni = rng.random(n) < 0.25
    P[uni] = rng.uniform(lo, hi, (int(uni.sum()), 3))
    P = np.clip(P, lo, hi)
    P[0] = lo
    P[1] = hi
    return P


def test_keys_at_cell_boundaries_and_far_bodies():
    """The tree kernels quantise each coordinate with one fused multiply-add
    and fall back to the exact FP64 formula within a bound of a cell
    boundary (a bound that grows with |lo| / (hi - lo)).  Beads on and one
    ulp beside cell boundaries, bodies far from the origin (up to 1e9 times
    their size, where every bead takes the exact formula), a body of size
    1e-6, and a body above the per-block sort limit (the device-wide key
    pass): every tree is bit-exact with the oracle's."""
    dev = _dev()
    zq = _zq()
    rng = np.random.default_rng(2024)
    pts = [
        _boundary_body(rng, 700, 0.0, 1.0),
        _boundary_body(rng, 900, -3.7, 37.0),
        _boundary_body(rng, 600, 1e6, 1.0),
        _boundary_body(rng, 600, -2.5e7, 3.0),
        _boundary_body(rng, 500, 1e9, 1.0),
        _boundary_body(rng, 400, 3.0, 1e-6),
        _boundary_body(rng, 1500, 12.0, 0.75),
        _boundary_body(rng, 9000, -40.0, 80.0),
    ]
    bt = _batch_from_points(pts)
    x, y, z = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (bt.x, bt.y, bt.z))
    ctx = zq.Context(0)
    ctx.build_tree_batched(bt.off, x, y, z, 6)
    check_tree(ctx, bt, oracle_bodies(bt))
    ctx.close()


def _batch_from_points(bodies_pts):
    off = np.zeros(len(bodies_pts) + 1, np.int64)
    off[1:] = np.cumsum([p.shape[0] for p in bodies_pts])
    P = np.concatenate(bodies_pts)
    return W.Batch(off, P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy())


@pytest.mark.parametrize("arith", ["dd", "fp64"])
def test_edge_geometries(arith):
    rng = np.random.default_rng(12)
    pts = [
        rng.uniform(-1, 1, (3, 3)),                                   # smallest body
        np.c_[rng.uniform(-1, 1, (40, 2)), np.full(40, 0.3)],         # flat (z = const)
        rng.uniform(-1, 1, (50, 3)) + [1e3, -2e3, 5e2],               # far from the origin
        np.c_[np.linspace(0, 1, 30), rng.normal(0, 1e-6, 30), rng.normal(0, 1e-6, 30)],  # near-collinear
        np.r_[rng.uniform(0, 1, (20, 3)), np.full((4, 3), 0.5)],      # beads sharing one cell
    ]
    bt = _batch_from_points(pts)
    ctx, _ = make_ctx(bt, cut=3, arith=arith)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    check_records(ctx, bt, bodies, arith, skip=(2,))
    check_apply(ctx, bt, np.float64)


@pytest.mark.parametrize("cluster", [20, 60])
def test_tight_clusters_sort_exactly(cluster):
    """A cluster of beads inside one cell of the first 10 2/3 octree levels
    (their keys share the high 32 bits) among spread-out beads: runs of at
    most 32 such beads are sorted by the fix-up, longer ones by the full
    sort; the tree is bit-exact either way.

    The sweeps are held to the conditioning of the input: a node's offset
    d = c_x - c_y between centroids of size |c| carries the last-bit
    rounding of the centroids (|c| 2^-53 each, in a different order of
    operations in the oracle and the kernels), so inside a cluster of extent
    delta the relative error of d, and of the rows of G built from it, is up
    to about 2 |c| 2^-53 / delta; the tolerance is 8 times that."""
    rng = np.random.default_rng(cluster)
    pts = [np.r_[rng.uniform(0, 1, (40, 3)), 0.5 + 1e-7 * rng.uniform(0, 1, (cluster, 3))],
           np.r_[rng.uniform(-3, 3, (900, 3)), 1.0 + 1e-6 * rng.uniform(0, 1, (cluster, 3))]]
    bt = _batch_from_points(pts)
    ctx, _ = make_ctx(bt, cut=3)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    tol = max(TOL[np.float64], 8 * 2 * 3.0 * 2.0 ** -53 / 1e-7)
    check_apply(ctx, bt, np.float64, tol=tol)


def test_coincident_beads_warn():
    rng = np.random.default_rng(1)
    p = rng.uniform(0, 1, (10, 3))
    p[7] = p[3]
    bt = _batch_from_points([p])
    zq = _zq()
    ctx, _ = make_ctx(bt, cut=3)
    assert ctx.sync(allow_degenerate=True) == zq.ZQ_WDEGENERATE
    check_tree(ctx, bt, oracle_bodies(bt))
    check_apply(ctx, bt, np.float64)


def test_non_finite_coordinates_reported():
    zq = _zq()
    bt = W.shell_body(64, seed=2)
    bt.x[5] = np.nan
    with pytest.raises(zq.ZQError) as ei:
        ctx, _ = make_ctx(bt, cut=3)
        ctx.sync()
    assert ei.value.code == zq.ZQ_ENONFINITE


def test_argument_errors():
    zq = _zq()
    dev = _dev()
    ctx = zq.Context(0)
    x = torch.zeros(2, dtype=torch.float64, device=dev)
    with pytest.raises(zq.ZQError) as ei:
        ctx.build_tree_batched(np.array([0, 2]), x, x, x)
    assert ei.value.code == zq.ZQ_EINVAL
    v = torch.zeros((3, 4), dtype=torch.float64, device=dev)
    with pytest.raises(zq.ZQError) as ei:
        ctx.apply_Q(v)
    assert ei.value.code == zq.ZQ_ESTATE


# --------------------------------------------------------- full sizes


@pytest.mark.parametrize("arith", ["dd", "fp64"])
def test_full_size_batched_shells(arith):
    """2000 bodies, log-uniform 50..5000 beads: every output against the
    oracle (FP32 and FP64 sweeps; transforms in double-single or FP64),
    tree bit-exact."""
    bt = W.shell_batch(m=2000, seed=0)
    ctx, _ = make_ctx(bt, arith=arith)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    del bodies
    check_apply(ctx, bt, np.float32, seed=7)
    check_apply(ctx, bt, np.float64, seed=7)


@pytest.mark.parametrize("arith", ["dd", "fp64"])
def test_full_size_ellipsoid(arith):
    """One body of 2^20 beads: tree bit-exact, sweeps against the oracle."""
    bt = W.ellipsoid_body(n=1 << 20, seed=0)
    ctx, _ = make_ctx(bt, arith=arith)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    del bodies
    check_apply(ctx, bt, np.float32, seed=9)
    check_apply(ctx, bt, np.float64, seed=9)


@pytest.mark.parametrize("arith", ["dd", "fp64"])
def test_collinear_and_lattice_bodies_match(arith):
    """Exactly collinear beads and lattice bodies (rank-deficient node
    matrices everywhere): the FP64 sweeps still match the oracle."""
    n = 30
    line = np.c_[np.arange(n) * 0.25, np.arange(n) * 0.5, np.full(n, 1.0)]
    g = np.arange(64)
    lattice = np.c_[g % 4, (g // 4) % 4, g // 16].astype(float) * 0.3
    bt = _batch_from_points([line, lattice])
    ctx, _ = make_ctx(bt, cut=3, arith=arith)
    bodies = oracle_bodies(bt)
    check_tree(ctx, bt, bodies)
    check_records(ctx, bt, bodies, arith)
    check_apply(ctx, bt, np.float64)
    check_apply(ctx, bt, np.float32)


@pytest.mark.parametrize("arith", ["dd", "fp64"])
def test_degenerate_warning_matches_oracle_flags(arith):
    """ZQ_WDEGENERATE is raised exactly for the batches in which the oracle
    flags a node (singular T22: collinear or coincident beads)."""
    zq = _zq()
    rng = np.random.default_rng(21)
    n = 24
    g = np.arange(n)
    cases = [
        [rng.uniform(0, 1, (50, 3)), rng.uniform(0, 1, (7, 3))],            # generic: no flag
        [np.c_[g * 0.5, g * 0.25, np.full(n, 2.0)]],                          # collinear
        [np.c_[g % 3, (g // 3) % 3, g // 9].astype(float)],                   # lattice
        [np.c_[np.linspace(0, 1, 30), rng.normal(0, 1e-6, 30), rng.normal(0, 1e-6, 30)]],
    ]
    for pts in cases:
        bt = _batch_from_points(pts)
        ctx, _ = make_ctx(bt, cut=2, arith=arith)
        want = any(B.node(q)["degenerate"] for B in oracle_bodies(bt) for q in range(B.n - 1))
        got = ctx.sync(allow_degenerate=True)
        assert got == (zq.ZQ_WDEGENERATE if want else zq.ZQ_OK), (pts[0][:2], want, got)
        ctx.close()
