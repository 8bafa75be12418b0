"""ctypes binding of libzq (include/zq.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module turns
torch tensors into device pointers and sizes, and C status codes into
exceptions.  The library must have been built (``__graft_entry__.build()``
or ``python paper_1708_08427_gb300/build.py``); importing this module
without it raises -- there is no CPU fallback.

Layouts (see include/zq.h): bead vectors are planes (k, 3, N) of the
caller's bead order; residue vectors are (k, R) with R = 3N - 6m.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libzq.so"

ZQ_OK, ZQ_EINVAL, ZQ_ENOMEM, ZQ_ECUDA, ZQ_ESTATE, ZQ_ENONFINITE, ZQ_WDEGENERATE = range(7)
ZQ_FP64, ZQ_FP32, ZQ_BF16, ZQ_TF32, ZQ_BF16_TC = 0, 1, 2, 3, 4
ZQ_HOST_BUFFERS, ZQ_KEEP_TREE, ZQ_GRAPH = 1, 2, 4
ZQ_BUILD_DD, ZQ_BUILD_FP64 = 0, 1
ZQ_STEP_LEVELS, ZQ_STEP_FUSED = 0, 1
ZQ_ORDER_CALLER, ZQ_ORDER_TREE = 0, 1
ZQ_ROWS_INORDER, ZQ_ROWS_PREORDER = 0, 1

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


class ZQError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_lib().zq_status_string(code).decode()} (status {code})")


_L: ctypes.CDLL | None = None


def _lib() -> ctypes.CDLL:
    global _L
    if _L is None:
        if not _LIB_PATH.exists():
            raise ImportError(f"libzq.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(str(_LIB_PATH))
        L.zq_status_string.restype = ctypes.c_char_p
        L.zq_status_string.argtypes = [ctypes.c_int]
        L.zq_create.restype = ctypes.c_int
        L.zq_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp]
        L.zq_destroy.restype = ctypes.c_int
        L.zq_destroy.argtypes = [_vp]
        L.zq_build_tree_batched.restype = ctypes.c_int
        L.zq_build_tree_batched.argtypes = [_vp, _i64, _i64p, _vp, _vp, _vp, ctypes.c_int32]
        L.zq_build_tree.restype = ctypes.c_int
        L.zq_build_tree.argtypes = [_vp, _i64, _vp, _vp, _vp, ctypes.c_int32]
        L.zq_build_transforms.restype = ctypes.c_int
        L.zq_build_transforms.argtypes = [_vp, _vp, _vp, _vp]
        for name in ("zq_apply_Q", "zq_apply_QT"):
            f = getattr(L, name)
            f.restype = ctypes.c_int
            f.argtypes = [_vp, ctypes.c_int, _i64, _vp, _i64, _vp, _i64]
        L.zq_sync.restype = ctypes.c_int
        L.zq_sync.argtypes = [_vp]
        L.zq_sizes.restype = ctypes.c_int
        L.zq_sizes.argtypes = [_vp, _i64p, _i64p, _i64p, _i64p]
        L.zq_get_tree.restype = ctypes.c_int
        L.zq_get_tree.argtypes = [_vp] + [_i32p] * 7
        L.zq_get_nodes.restype = ctypes.c_int
        L.zq_get_nodes.argtypes = [_vp, _f64p, _f64p]
        L.zq_get_records.restype = ctypes.c_int
        L.zq_get_records.argtypes = [_vp, _f64p]
        L.zq_pipeline.restype = ctypes.c_int
        L.zq_pipeline.argtypes = [_vp, ctypes.c_int, _i64, _i64p, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                  ctypes.c_int32, ctypes.c_int32]
        L.zq_time_kernel.restype = ctypes.c_int
        L.zq_time_kernel.argtypes = [_vp, ctypes.c_char_p, _vp, _vp]
        L.zq_set_build_arith.restype = ctypes.c_int
        L.zq_set_build_arith.argtypes = [_vp, ctypes.c_int]
        L.zq_set_step_schedule.restype = ctypes.c_int
        L.zq_set_step_schedule.argtypes = [_vp, ctypes.c_int]
        L.zq_set_vector_order.restype = ctypes.c_int
        L.zq_set_vector_order.argtypes = [_vp, ctypes.c_int]
        L.zq_launch_count.restype = ctypes.c_int
        L.zq_launch_count.argtypes = [_vp, _i64p]
        L.zq_apply_Q_full.restype = ctypes.c_int
        L.zq_apply_Q_full.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
        L.zq_apply_QT_full.restype = ctypes.c_int
        L.zq_apply_QT_full.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp]
        L.zq_apply_pair.restype = ctypes.c_int
        L.zq_apply_pair.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.zq_apply_rotated.restype = ctypes.c_int
        L.zq_qgen_nnz.restype = ctypes.c_int
        L.zq_qgen_nnz.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
        L.zq_qgen.restype = ctypes.c_int
        L.zq_qgen.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.zq_apply_rotated.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
        L.zq_reserve_block.restype = ctypes.c_int
        L.zq_reserve_block.argtypes = [_vp, ctypes.c_int, _i64]
        for name in ("zq_apply_Q_block", "zq_apply_QT_block"):
            f = getattr(L, name)
            f.restype = ctypes.c_int
            f.argtypes = [_vp, ctypes.c_int, _i64, _vp, _vp]
        L.zq_residue_offsets.restype = ctypes.c_int
        L.zq_residue_offsets.argtypes = [_i64, _i64p, _i32p, _i32p, ctypes.c_int, _i64p, _i64p]
        L.zq_get_residue_offsets.restype = ctypes.c_int
        L.zq_get_residue_offsets.argtypes = [_vp, ctypes.c_int, _i64p, _i64p]
        L.zq_apply_Q_noalloc.restype = ctypes.c_int
        L.zq_apply_Q_noalloc.argtypes = [ctypes.c_int, _vp, _i64, _vp, _vp, _vp, _vp, _vp]
        _L = L
    return _L


def library_path() -> Path:
    return _LIB_PATH


def _check(code: int, where: str, allow=(ZQ_OK,)):
    if code not in allow:
        raise ZQError(code, where)
    return code


def _ptr(t) -> int:
    return int(t.data_ptr())


def _np_i32(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_i32p)


class Context:
    """Owns a zq_ctx: tree, transforms and scratch on one device/stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self._torch = torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = _vp()
        _check(_lib().zq_create(ctypes.byref(h), device, _vp(stream.cuda_stream)), "zq_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().zq_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ builds
    def build_tree_batched(self, off, x, y, z, level_cut: int = 0):
        off = np.ascontiguousarray(off, dtype=np.int64)
        self._off = off
        m = off.shape[0] - 1
        for t in (x, y, z):
            assert t.is_cuda and t.dtype == self._torch.float64 and t.is_contiguous()
        _check(_lib().zq_build_tree_batched(self._h, m, off.ctypes.data_as(_i64p), _ptr(x), _ptr(y),
                                            _ptr(z), int(level_cut)), "zq_build_tree_batched")

    def build_tree(self, x, y, z, level_cut: int = 0):
        self.build_tree_batched(np.array([0, x.shape[0]], np.int64), x, y, z, level_cut)

    def build_transforms(self, x, y, z):
        _check(_lib().zq_build_transforms(self._h, _ptr(x), _ptr(y), _ptr(z)), "zq_build_transforms")

    # ------------------------------------------------------------ applies
    def sizes(self):
        N, m, R, nodes = _i64(), _i64(), _i64(), _i64()
        _check(_lib().zq_sizes(self._h, ctypes.byref(N), ctypes.byref(m), ctypes.byref(R),
                               ctypes.byref(nodes)), "zq_sizes")
        return int(N.value), int(m.value), int(R.value), int(nodes.value)

    @staticmethod
    def _prec(t):
        import torch

        if t.dtype == torch.float64:
            return ZQ_FP64
        if t.dtype == torch.float32:
            return ZQ_FP32
        raise TypeError("vectors must be float32 or float64")

    def apply_Q(self, v, out=None):
        """v: (3, N) or (k, 3, N) device tensor -> (R,) or (k, R)."""
        N, m, R, _ = self.sizes()
        squeeze = v.dim() == 2
        vv = v.reshape(-1, 3 * N)
        assert vv.is_contiguous() and v.is_cuda
        k = vv.shape[0]
        if out is None:
            out = self._torch.empty((k, R), dtype=v.dtype, device=v.device)
        oo = out.reshape(k, R)
        _check(_lib().zq_apply_Q(self._h, self._prec(v), k, _ptr(vv), 3 * N, _ptr(oo), R), "zq_apply_Q")
        return out.reshape(R) if squeeze and out.dim() == 2 else out

    def apply_Q_full(self, v, out=None, root=None):
        """Q~ v (R,) and the root Info-sets Q_Z v per body (m, 6); v: (3, N)."""
        N, m, R, _ = self.sizes()
        assert v.is_cuda and v.is_contiguous() and v.numel() == 3 * N
        if out is None:
            out = self._torch.empty(R, dtype=v.dtype, device=v.device)
        if root is None:
            root = self._torch.empty((m, 6), dtype=v.dtype, device=v.device)
        _check(_lib().zq_apply_Q_full(self._h, self._prec(v), _ptr(v), _ptr(out), _ptr(root)), "zq_apply_Q_full")
        return out, root

    def apply_QT_full(self, w, root, out=None):
        """Q~^T w + Q_Z^T root -> (3, N); w: (R,), root: (m, 6)."""
        N, m, R, _ = self.sizes()
        assert w.is_cuda and w.is_contiguous() and w.numel() == R
        assert root.is_cuda and root.is_contiguous() and root.numel() == 6 * m and root.dtype == w.dtype
        if out is None:
            out = self._torch.empty((3, N), dtype=w.dtype, device=w.device)
        _check(_lib().zq_apply_QT_full(self._h, self._prec(w), _ptr(w), _ptr(root), _ptr(out)),
               "zq_apply_QT_full")
        return out

    def apply_pair(self, v, w, qv=None, qtw=None):
        """Q~ v and Q~^T w together (concurrent sweeps): v (3, N), w (R,)."""
        N, m, R, _ = self.sizes()
        assert v.is_cuda and w.is_cuda and v.dtype == w.dtype and v.numel() == 3 * N and w.numel() == R
        assert v.is_contiguous() and w.is_contiguous()
        if qv is None:
            qv = self._torch.empty(R, dtype=v.dtype, device=v.device)
        if qtw is None:
            qtw = self._torch.empty((3, N), dtype=v.dtype, device=v.device)
        _check(_lib().zq_apply_pair(self._h, self._prec(v), _ptr(v), _ptr(qv), _ptr(w), _ptr(qtw)),
               "zq_apply_pair")
        return qv, qtw

    def apply_rotated(self, Rm, v=None, w=None, qv=None, qtw=None):
        """Products for rigidly moved bodies on the transforms built for the
        reference coordinates: Q~ blockdiag(R_j^T) v and blockdiag(R_j) Q~^T w.
        Rm: (m, 3, 3) or (m, 9) float64 CUDA rotations; v (3, N), w (R,) of one
        dtype (either may be None).  Returns (qv, qtw), None for a skipped one."""
        import torch

        N, m, R, _ = self.sizes()
        assert Rm.is_cuda and Rm.dtype == torch.float64 and Rm.is_contiguous() and Rm.numel() == 9 * m
        assert v is not None or w is not None
        ref = v if v is not None else w
        if v is not None:
            assert v.is_cuda and v.is_contiguous() and v.numel() == 3 * N
            if qv is None:
                qv = torch.empty(R, dtype=v.dtype, device=v.device)
        if w is not None:
            assert w.is_cuda and w.is_contiguous() and w.numel() == R and w.dtype == ref.dtype
            if qtw is None:
                qtw = torch.empty((3, N), dtype=w.dtype, device=w.device)
        p = lambda t: _ptr(t) if t is not None else None
        _check(_lib().zq_apply_rotated(self._h, self._prec(ref), _ptr(Rm), p(v), p(qv), p(w), p(qtw)),
               "zq_apply_rotated")
        return (qv if v is not None else None), (qtw if w is not None else None)

    def qgen_nnz(self) -> int:
        """Nonzeros of the explicit Q~ (synchronises the context stream)."""
        n = ctypes.c_int64()
        _check(_lib().zq_qgen_nnz(self._h, ctypes.byref(n)), "zq_qgen_nnz")
        return int(n.value)

    def qgen(self, dtype=None, with_u: bool = False, device=None):
        """The explicit Q~ as CSR arrays (row_ptr int64 (R+1), col int32,
        val): columns 3 i + a in the caller's bead order.  with_u: also the
        rotational rows U_j of Q_Z, 9 N values (body j's 3 x 3 n_j block at
        9 off[j]).  Returns (row_ptr, col, val, U or None)."""
        import torch

        dtype = dtype or torch.float64
        dev = device or torch.device("cuda", self.device)
        N, m, R, _ = self.sizes()
        nnz = self.qgen_nnz()
        row_ptr = torch.empty(R + 1, dtype=torch.int64, device=dev)
        col = torch.empty(nnz, dtype=torch.int32, device=dev)
        val = torch.empty(nnz, dtype=dtype, device=dev)
        U = torch.empty(9 * N, dtype=dtype, device=dev) if with_u else None
        return self.qgen_into(row_ptr, col, val, U)

    def qgen_into(self, row_ptr, col, val, U=None):
        """zq_qgen into given device buffers (sizes as qgen's results)."""
        import torch

        p = {torch.float64: ZQ_FP64, torch.float32: ZQ_FP32}[val.dtype]
        assert row_ptr.dtype == torch.int64 and col.dtype == torch.int32 and (U is None or U.dtype == val.dtype)
        _check(_lib().zq_qgen(self._h, p, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(U) if U is not None else None),
               "zq_qgen")
        return row_ptr, col, val, U

    # ------------------------------------------------------- block form
    @staticmethod
    def _bprec(t, tensor_cores: bool = False):
        import torch

        if tensor_cores:
            return {torch.float32: ZQ_TF32, torch.bfloat16: ZQ_BF16_TC}[t.dtype]
        return {torch.float64: ZQ_FP64, torch.float32: ZQ_FP32, torch.bfloat16: ZQ_BF16}[t.dtype]

    def reserve_block(self, k_max: int, dtype):
        """Block scratch for up to k_max columns of this dtype (the same
        scratch serves the tensor-core forms of float32 and bfloat16)."""
        import torch

        p = {torch.float64: ZQ_FP64, torch.float32: ZQ_FP32, torch.bfloat16: ZQ_BF16}[dtype]
        _check(_lib().zq_reserve_block(self._h, p, int(k_max)), "zq_reserve_block")

    def apply_Q_block(self, V, out=None, tensor_cores: bool = False):
        """V: (3N, k) device tensor (rows of k; row a*N + i) -> (R, k).
        tensor_cores: the node products on tensor cores (float32: ZQ_TF32,
        bfloat16: ZQ_BF16_TC)."""
        N, m, R, _ = self.sizes()
        assert V.is_cuda and V.is_contiguous() and V.dim() == 2 and V.shape[0] == 3 * N
        k = V.shape[1]
        if out is None:
            out = self._torch.empty((R, k), dtype=V.dtype, device=V.device)
        assert out.is_contiguous() and tuple(out.shape) == (R, k) and out.dtype == V.dtype
        _check(_lib().zq_apply_Q_block(self._h, self._bprec(V, tensor_cores), k, _ptr(V), _ptr(out)),
               "zq_apply_Q_block")
        return out

    def apply_QT_block(self, W, out=None, tensor_cores: bool = False):
        """W: (R, k) device tensor -> (3N, k); tensor_cores as apply_Q_block."""
        N, m, R, _ = self.sizes()
        assert W.is_cuda and W.is_contiguous() and W.dim() == 2 and W.shape[0] == R
        k = W.shape[1]
        if out is None:
            out = self._torch.empty((3 * N, k), dtype=W.dtype, device=W.device)
        assert out.is_contiguous() and tuple(out.shape) == (3 * N, k) and out.dtype == W.dtype
        _check(_lib().zq_apply_QT_block(self._h, self._bprec(W, tensor_cores), k, _ptr(W), _ptr(out)),
               "zq_apply_QT_block")
        return out

    def apply_QT(self, w, out=None):
        """w: (R,) or (k, R) device tensor -> (3, N) or (k, 3, N)."""
        N, m, R, _ = self.sizes()
        squeeze = w.dim() == 1
        ww = w.reshape(-1, R)
        assert ww.is_contiguous() and w.is_cuda
        k = ww.shape[0]
        if out is None:
            out = self._torch.empty((k, 3, N), dtype=w.dtype, device=w.device)
        _check(_lib().zq_apply_QT(self._h, self._prec(w), k, _ptr(ww), R, _ptr(out), 3 * N), "zq_apply_QT")
        return out.reshape(3, N) if squeeze else out

    def pipeline(self, off, x, y, z, v=None, qv=None, w=None, qtw=None, level_cut: int = 0,
                 host: bool = False, keep_tree: bool = False, prec: int | None = None, graph: bool = False):
        """One step: tree, FP64 transforms, qv = Q~ v, qtw = Q~^T w.  With
        host=True all tensors are (pinned) host tensors staged by the
        library; otherwise device tensors.  off: numpy int64 (m + 1).
        graph=True: the library captures the step as a CUDA graph and
        replays it while the arguments are unchanged (ZQ_GRAPH)."""
        off = np.ascontiguousarray(off, dtype=np.int64)
        self._off = off
        m = off.shape[0] - 1
        ref = v if v is not None else w
        if prec is None:
            prec = self._prec(ref)
        flags = (ZQ_HOST_BUFFERS if host else 0) | (ZQ_KEEP_TREE if keep_tree else 0) | (ZQ_GRAPH if graph else 0)
        p = lambda t: None if t is None else _ptr(t)
        _check(_lib().zq_pipeline(self._h, prec, m, off.ctypes.data_as(_i64p), _ptr(x), _ptr(y), _ptr(z),
                                  p(v), p(qv), p(w), p(qtw), int(level_cut), flags), "zq_pipeline")

    def time_kernel(self, name: str | None, start=None, stop=None):
        """Bracket launches of kernel `name` with torch.cuda.Event start/stop
        (events must have been recorded once so their handles exist)."""
        if name is None:
            _check(_lib().zq_time_kernel(self._h, None, None, None), "zq_time_kernel")
            return
        _check(_lib().zq_time_kernel(self._h, name.encode(), _vp(start.cuda_event), _vp(stop.cuda_event)),
               "zq_time_kernel")

    def set_vector_order(self, order: str):
        """'caller' (default) or 'tree': bead vectors of the products in the
        tree's sorted-position order (entry s = caller's bead perm[s])."""
        _check(_lib().zq_set_vector_order(self._h, {"caller": ZQ_ORDER_CALLER, "tree": ZQ_ORDER_TREE}[order]), "zq_set_vector_order")

    def set_step_schedule(self, schedule: str):
        """zq_set_step_schedule: "levels" or "fused" (include/zq.h)."""
        code = {"levels": ZQ_STEP_LEVELS, "fused": ZQ_STEP_FUSED}[schedule]
        _check(_lib().zq_set_step_schedule(self._h, code), "zq_set_step_schedule")

    def set_build_arith(self, arith: str):
        """'dd' (double-single on the FP32 pipes, default) or 'fp64'."""
        code = {"dd": ZQ_BUILD_DD, "fp64": ZQ_BUILD_FP64}[arith]
        _check(_lib().zq_set_build_arith(self._h, code), "zq_set_build_arith")

    def launch_count(self) -> int:
        n = _i64()
        _check(_lib().zq_launch_count(self._h, ctypes.byref(n)), "zq_launch_count")
        return int(n.value)

    def sync(self, allow_degenerate: bool = False):
        allow = (ZQ_OK, ZQ_WDEGENERATE) if allow_degenerate else (ZQ_OK,)
        return _check(_lib().zq_sync(self._h), "zq_sync", allow)

    # ------------------------------------------------------------ exports
    def get_tree(self) -> dict:
        N, m, R, nodes = self.sizes()
        perm = np.empty(N, np.int32)
        arrs = {k: np.empty(nodes, np.int32) for k in ("left", "right", "first", "count", "height", "roff")}
        _check(_lib().zq_get_tree(self._h, _np_i32(perm), _np_i32(arrs["left"]), _np_i32(arrs["right"]),
                                  _np_i32(arrs["first"]), _np_i32(arrs["count"]), _np_i32(arrs["height"]),
                                  _np_i32(arrs["roff"])), "zq_get_tree")
        return dict(perm=perm, **arrs)

    def residue_offsets(self, order: str = "preorder"):
        """Per-node residue offsets of the current tree in row order
        'inorder' (the products' order) or 'preorder' (the recursive layout
        [Residue_p; diag(Q~_x, Q~_y)]); returns (node_off, body_off), int64."""
        N, m, R, nodes = self.sizes()
        node_off = np.empty(nodes, np.int64)
        body_off = np.empty(m + 1, np.int64)
        _check(_lib().zq_get_residue_offsets(self._h, _ROW_ORDER[order], node_off.ctypes.data_as(_i64p),
                                             body_off.ctypes.data_as(_i64p)), "zq_get_residue_offsets")
        return node_off, body_off

    def get_nodes(self):
        N, m, R, nodes = self.sizes()
        c = np.empty((nodes, 3))
        L = np.empty((nodes, 6))
        _check(_lib().zq_get_nodes(self._h, c.ctypes.data_as(_f64p), L.ctypes.data_as(_f64p)),
               "zq_get_nodes")
        return c, L

    def get_records(self) -> np.ndarray:
        """FP64 node records, shape (nodes, 28) (layout in include/zq.h)."""
        N, m, R, nodes = self.sizes()
        rec = np.empty((nodes, 28))
        _check(_lib().zq_get_records(self._h, rec.ctypes.data_as(_f64p)), "zq_get_records")
        return rec


ZQ_NOALLOC_MAX_BEADS = 2048


_ROW_ORDER = {"inorder": ZQ_ROWS_INORDER, "preorder": ZQ_ROWS_PREORDER}


def residue_offsets(off, left, right, order: str = "preorder"):
    """zq_residue_offsets on host arrays in zq_get_tree's form: off (m + 1)
    bead offsets, left / right child codes of the N - m internal nodes.
    Returns (node_off, body_off), int64."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    left = np.ascontiguousarray(left, dtype=np.int32)
    right = np.ascontiguousarray(right, dtype=np.int32)
    m = off.shape[0] - 1
    node_off = np.empty(left.shape[0], np.int64)
    body_off = np.empty(m + 1, np.int64)
    assert right.shape == left.shape and m >= 1 and left.shape[0] == int(off[-1]) - m
    _check(_lib().zq_residue_offsets(m, off.ctypes.data_as(_i64p), _np_i32(left), _np_i32(right),
                                     _ROW_ORDER[order], node_off.ctypes.data_as(_i64p),
                                     body_off.ctypes.data_as(_i64p)), "zq_residue_offsets")
    return node_off, body_off


def apply_Q_noalloc(x, y, z, v, out, stream=None):
    """Q~v for one body of 3..ZQ_NOALLOC_MAX_BEADS beads through
    zq_apply_Q_noalloc (no device allocation in the library; the caller
    provides every buffer).  x, y, z: (n,) float64 device tensors; v: (3, n)
    float64 device planes; out: (3n - 6,) float64 device tensor."""
    import torch

    n = int(x.numel())
    if not 3 <= n <= ZQ_NOALLOC_MAX_BEADS:
        raise ValueError(f"zq_apply_Q_noalloc takes 3..{ZQ_NOALLOC_MAX_BEADS} beads, got {n}")
    for t in (x, y, z, v, out):
        assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    assert v.numel() == 3 * n and out.numel() == 3 * n - 6
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    _check(_lib().zq_apply_Q_noalloc(x.device.index, _vp(stream.cuda_stream), n, _ptr(x), _ptr(y),
                                      _ptr(z), _ptr(v), _ptr(out)), "zq_apply_Q_noalloc")
    return out


# raw C entry points, same names as include/zq.h
def __getattr__(name):
    if name.startswith("zq_"):
        return getattr(_lib(), name)
    raise AttributeError(name)
