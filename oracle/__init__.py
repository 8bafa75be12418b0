"""FP64 CPU oracle for Q~v / Q~^T w (arXiv 1708.08427) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps the plain C implementation
in ``zq_oracle.c`` through ctypes and shares no code with the CUDA library.

Vectors follow the paper's ordering f = [f_1; ...; f_n] (component 3i + a is
axis a of bead i); residues follow the node order of the split position,
bodies concatenated (Sec. 1: Q~ = diag(Q~^1, ..., Q~^m)).

Parity status of each function (pins live in tests/test_oracle_*.py):
  tree            pinned: brute-force bisection on tiny inputs, an
                  independent sort-and-prefix construction, invariants.
  lq              pinned: LAPACK dgeqrf/dorgqr via numpy.linalg.qr (the
                  paper computes Eq. 3.5 with Matlab qr, which is LAPACK),
                  with R's diagonal made nonnegative (unique for full rank).
  degenerate      pinned: the singular-T22 flag equals exact collinearity
                  of the node's beads on integer lattices.
  case_one        pinned: the printed closed form, Eqs. 3.9-3.10.
  apply_Q/_QT     pinned: dense projector I - Z^T (Z Z^T)^{-1} Z, SVD
                  complement, rigid-field annihilation, Parseval,
                  force/torque-free outputs, round trips (Table 1).
  qgen            pinned: Q Q^T = I, Q Z^T = 0 and agreement with the
                  implicit passes (Table 1 columns 2-7).
  batch_apply_rotated
                  pinned: for bodies moved rigidly, the moved body's Z
                  (Eq. 1.2, from the moved coordinates) annihilates the
                  rows, the rows stay orthonormal, Q~^T Q~ is the moved
                  body's projector, and R = I gives batch_apply exactly.
  residue basis   rows 4..k of G are the LAPACK completion; the paper fixes
                  them only through "Matlab qr", so they are pinned exactly
                  as far as LAPACK is, and otherwise only through the
                  basis-free projector checks above.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "zq_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libzq_oracle.so"

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int32_p = ctypes.POINTER(ctypes.c_int32)
_c_int64_p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False, src: Path | None = None, out: Path | None = None) -> Path:
    """Compile the oracle with gcc (no FMA contraction, FP64 throughout)."""
    src = Path(src) if src else _SRC
    out = Path(out) if out else _LIB_PATH
    if not force and out.exists() and out.stat().st_mtime >= src.stat().st_mtime:
        return out
    out.parent.mkdir(parents=True, exist_ok=True)
    tmp = out.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           str(src), "-lm", "-o", str(tmp)]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    lib.orc_body_new.restype = ctypes.c_void_p
    lib.orc_body_new.argtypes = [ctypes.c_int64, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_body_free.restype = None
    lib.orc_body_free.argtypes = [ctypes.c_void_p]
    lib.orc_body_n.restype = ctypes.c_int64
    lib.orc_body_n.argtypes = [ctypes.c_void_p]
    lib.orc_body_tree.restype = None
    lib.orc_body_tree.argtypes = [ctypes.c_void_p] + [_c_int32_p] * 6 + [_c_int64_p, _c_int32_p]
    lib.orc_body_node.restype = None
    lib.orc_body_node.argtypes = [ctypes.c_void_p, ctypes.c_int64, _c_int32_p, _c_int32_p,
                                  _c_int32_p, _c_double_p, _c_double_p, _c_double_p,
                                  _c_double_p]
    lib.orc_body_nodes_all.restype = None
    lib.orc_body_nodes_all.argtypes = [ctypes.c_void_p, _c_double_p, _c_double_p]
    lib.orc_lq.restype = None
    lib.orc_lq.argtypes = [_c_double_p, ctypes.c_int32, _c_double_p, _c_double_p]
    lib.orc_case_one.restype = None
    lib.orc_case_one.argtypes = [_c_double_p, ctypes.c_double, _c_double_p, _c_double_p,
                                 _c_int32_p]
    lib.orc_body_apply_Q.restype = None
    lib.orc_body_apply_Q.argtypes = [ctypes.c_void_p, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_body_apply_QT.restype = None
    lib.orc_body_apply_QT.argtypes = [ctypes.c_void_p, _c_double_p, _c_double_p, _c_double_p]
    lib.orc_body_qgen.restype = None
    lib.orc_body_qgen.argtypes = [ctypes.c_void_p, _c_double_p, _c_double_p]
    lib.orc_batch_apply.restype = ctypes.c_int
    lib.orc_batch_apply.argtypes = [ctypes.c_int64, _c_int64_p, _c_double_p, _c_double_p,
                                    _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                    _c_double_p]
    return lib


_LIB: ctypes.CDLL | None = None


def load(path: Path | None = None) -> ctypes.CDLL:
    """Load the oracle library (building it first if needed).  A path other
    than the default loads that build instead (used by the mutation tests)."""
    global _LIB
    if path is not None:
        return _bind(ctypes.CDLL(str(path)))
    if _LIB is None:
        _LIB = _bind(ctypes.CDLL(str(build())))
    return _LIB


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_c_double_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Body:
    """One rigid body: tree + node transforms built at construction."""

    def __init__(self, x, y, z, lib: ctypes.CDLL | None = None):
        self._lib = lib or load()
        self.x, self.y, self.z = _f64(x), _f64(y), _f64(z)
        self.n = int(self.x.shape[0])
        if self.n < 3:
            raise ValueError("a rigid body needs at least 3 beads")
        h = self._lib.orc_body_new(self.n, _dp(self.x), _dp(self.y), _dp(self.z))
        if not h:
            raise MemoryError("oracle body construction failed")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_body_free(h)
            self._h = None

    def tree(self) -> dict:
        n = self.n
        perm = np.empty(n, np.int32)
        arrs = {k: np.empty(n - 1, np.int32) for k in ("left", "right", "first", "last", "height")}
        roff = np.empty(n - 1, np.int64)
        root = ctypes.c_int32()
        self._lib.orc_body_tree(self._h, perm.ctypes.data_as(_c_int32_p),
                                *(arrs[k].ctypes.data_as(_c_int32_p)
                                  for k in ("left", "right", "first", "last", "height")),
                                roff.ctypes.data_as(_c_int64_p), ctypes.byref(root))
        return dict(perm=perm, roff=roff, root=int(root.value), **arrs)

    def node(self, g: int) -> dict:
        k, cnt, dg = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ab, c, L, G = np.empty(2), np.empty(3), np.empty(9), np.empty(81)
        self._lib.orc_body_node(self._h, int(g), ctypes.byref(k), ctypes.byref(cnt),
                                ctypes.byref(dg), _dp(ab), _dp(c), _dp(L), _dp(G))
        kk = int(k.value)
        return dict(k=kk, cnt=int(cnt.value), degenerate=bool(dg.value), alpha=ab[0],
                    beta=ab[1], c=c, L=L.reshape(3, 3), G=G[:kk * kk].reshape(kk, kk))

    def nodes_all(self):
        """(T22, centroid) of every node by split position: (n-1, 3, 3) lower
        triangular and (n-1, 3)."""
        L = np.empty((self.n - 1) * 9)
        c = np.empty((self.n - 1) * 3)
        self._lib.orc_body_nodes_all(self._h, _dp(L), _dp(c))
        return L.reshape(self.n - 1, 3, 3), c.reshape(self.n - 1, 3)

    def apply_Q(self, f, with_root: bool = False):
        f = _f64(f)
        assert f.shape == (3 * self.n,)
        out = np.empty(3 * self.n - 6)
        root = np.empty(6)
        self._lib.orc_body_apply_Q(self._h, _dp(f), _dp(out), _dp(root))
        return (out, root) if with_root else out

    def apply_QT(self, w, root6=None):
        w = _f64(w)
        assert w.shape == (3 * self.n - 6,)
        out = np.empty(3 * self.n)
        r = None if root6 is None else _f64(root6)
        self._lib.orc_body_apply_QT(self._h, _dp(w), None if r is None else _dp(r), _dp(out))
        return out

    def qgen(self):
        n3 = 3 * self.n
        Qt = np.empty((n3 - 6, n3))
        QZ = np.empty((6, n3))
        self._lib.orc_body_qgen(self._h, _dp(Qt), _dp(QZ))
        return Qt, QZ


def lq(M, lib: ctypes.CDLL | None = None):
    """LQ of a 3 x k matrix (Eq. 3.5): returns (L 3x3, G k x k)."""
    lib = lib or load()
    M = _f64(M)
    k = M.shape[1]
    L, G = np.empty(9), np.empty(k * k)
    lib.orc_lq(_dp(M), k, _dp(L), _dp(G))
    return L.reshape(3, 3), G.reshape(k, k)


def case_one(d, sk, lib: ctypes.CDLL | None = None):
    """Case I node (Eqs. 3.9-3.10): returns (T22, G, degenerate)."""
    lib = lib or load()
    d = _f64(d)
    L, G = np.empty(9), np.empty(9)
    dg = ctypes.c_int32()
    lib.orc_case_one(_dp(d), float(sk), _dp(L), _dp(G), ctypes.byref(dg))
    return L.reshape(3, 3), G.reshape(3, 3), bool(dg.value)


def batch_apply(off, x, y, z, f=None, w=None, lib: ctypes.CDLL | None = None):
    """Q~ f and Q~^T w over many bodies (interleaved bead vectors)."""
    lib = lib or load()
    off = np.ascontiguousarray(off, dtype=np.int64)
    m = off.shape[0] - 1
    N = int(off[-1])
    x, y, z = _f64(x), _f64(y), _f64(z)
    R = 3 * N - 6 * m
    qf = np.empty(R) if f is not None else None
    qtw = np.empty(3 * N) if w is not None else None
    fa = None if f is None else _f64(f)
    wa = None if w is None else _f64(w)
    rc = lib.orc_batch_apply(m, off.ctypes.data_as(_c_int64_p), _dp(x), _dp(y), _dp(z),
                             None if fa is None else _dp(fa), None if qf is None else _dp(qf),
                             None if wa is None else _dp(wa), None if qtw is None else _dp(qtw))
    if rc != 0:
        raise ValueError("oracle batch failed (a body with < 3 beads?)")
    return qf, qtw


def batch_apply_rotated(off, x, y, z, Rm, f=None, w=None, lib: ctypes.CDLL | None = None):
    """Q~ f and Q~^T w of bodies moved rigidly from (x, y, z): body j's beads
    taken to R_j r + d_j.  From Z's definition (Sec. 1, Eq. 1.2),
    Z_moved blockdiag(R_j) = diag(R_j, R_j) Z, so Q~ blockdiag(R_j^T) is an
    orthonormal complement of the moved body's Z rows.  Each bead vector of
    f is rotated by R_j^T before Q~; each bead vector of Q~^T w is rotated by
    R_j after.  Rm: (m, 3, 3); f, w, results as batch_apply."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    Rm = np.asarray(Rm, dtype=np.float64).reshape(-1, 3, 3)
    N = int(off[-1])
    body = np.repeat(np.arange(off.shape[0] - 1), np.diff(off))
    fr = None
    if f is not None:
        fb = _f64(f).reshape(N, 3)
        fr = np.einsum("nba,nb->na", Rm[body], fb).reshape(-1)     # R_j^T f_i
    qf, qtw = batch_apply(off, x, y, z, fr, w, lib)
    if qtw is not None:
        qtw = np.einsum("nab,nb->na", Rm[body], qtw.reshape(N, 3)).reshape(-1)  # R_j u_i
    return qf, qtw
