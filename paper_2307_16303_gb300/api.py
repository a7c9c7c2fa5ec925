"""Thin ctypes binding over libh3d.so (C ABI in include/h3d.h).

Argument marshalling only: every step of the build and of the product runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  If
the library has not been built, loading raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libh3d.so")

KERNELS = {"laplace": 0, "yukawa": 1, "inv_r4": 2, "cos_r": 3}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_3xtf32": 2}
ADMISSIBILITY = {"hodlr3d": 0, "strong": 1, "weak": 2}
STORAGE = {"factors": 0, "skeleton": 1, "symmetric": 2}
STATUS_NAMES = {0: "H3D_OK", 1: "H3D_ERR_ARG", 2: "H3D_ERR_DOMAIN", 3: "H3D_ERR_OOM", 4: "H3D_ERR_CUDA",
                5: "H3D_ERR_ACA_RANK", 6: "H3D_ERR_TIMEOUT", 7: "H3D_ERR_STATE", 8: "H3D_ERR_DEPTH"}

# every entry point declared in include/h3d.h
EXPORTS = ("h3d_default_options", "h3d_build", "h3d_matvec", "h3d_matvec_T", "h3d_matvec_host", "h3d_free",
           "h3d_status_string", "h3d_get_stats", "h3d_matvec_profile", "h3d_export_tree", "h3d_export_lists",
           "h3d_export_pivots", "h3d_import_pivots", "h3d_set_points", "h3d_debug_fail_alloc",
           "h3d_morton_order_noalloc", "h3d_energy", "h3d_forces",
           "h3d_batch_create", "h3d_batch_matvec", "h3d_batch_tune", "h3d_batch_configure", "h3d_batch_info",
           "h3d_batch_queue", "h3d_batch_groups", "h3d_batch_set_wait_limit", "h3d_batch_get_queue", "h3d_batch_set_queue",
           "h3d_batch_free")


class H3DError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        msg = lib().h3d_status_string(status).decode()
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)} ({msg})")
        self.status = status


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("kappa", C.c_double), ("rank_cap", C.c_int),
                ("lo", C.c_double * 3), ("side", C.c_double), ("workspace_bytes", C.c_int64),
                ("admissibility", C.c_int), ("storage", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("N", C.c_int64), ("depth", C.c_int), ("precision", C.c_int), ("kernel", C.c_int),
                ("leaf_size", C.c_int), ("tol", C.c_double), ("n_boxes", C.c_int64), ("n_leaves", C.c_int64),
                ("n_blocks", C.c_int64), ("n_vertex_blocks", C.c_int64), ("n_near", C.c_int64),
                ("max_rank", C.c_int), ("sum_rank", C.c_int64), ("factor_entries", C.c_int64),
                ("u_entries", C.c_int64), ("v_entries", C.c_int64),
                ("factor_bytes", C.c_int64), ("near_interactions", C.c_int64), ("device_bytes", C.c_int64),
                ("build_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libh3d.so; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libh3d.so not built ({LIB_PATH}); run paper_2307_16303_gb300.build_ext.build()")
        L = C.CDLL(LIB_PATH)
        P, i64, i32, f64 = C.c_void_p, C.c_int64, C.c_int, C.c_double
        sig = {
            "h3d_default_options": (None, [C.POINTER(Options)]),
            "h3d_build": (i32, [P, i64, i32, i32, f64, C.POINTER(Options), P, C.POINTER(P)]),
            "h3d_matvec": (i32, [P, P, P, i32, P]),
            "h3d_matvec_T": (i32, [P, P, P, i32, P]),
            "h3d_matvec_host": (i32, [P, P, P, i32, P]),
            "h3d_free": (i32, [P]),
            "h3d_status_string": (C.c_char_p, [i32]),
            "h3d_get_stats": (i32, [P, C.POINTER(Stats)]),
            "h3d_matvec_profile": (i32, [P, P, P, i32, P, C.POINTER(C.c_float), i32]),
            "h3d_export_tree": (i32, [P, P, P, P, P, P, P]),
            "h3d_export_lists": (i32, [P, P, P, P, P, P, P, P]),
            "h3d_export_pivots": (i32, [P, P, P, P]),
            "h3d_import_pivots": (i32, [P, P, P, P, P]),
            "h3d_set_points": (i32, [P, P, P]),
            "h3d_debug_fail_alloc": (None, [i64]),
            "h3d_morton_order_noalloc": (i32, [P, i64, P, f64, P, P, P]),
            "h3d_energy": (i32, [P, P, P, P, P]),
            "h3d_forces": (i32, [P, P, P, P, P]),
            "h3d_batch_create": (i32, [P, i32, C.POINTER(P)]),
            "h3d_batch_matvec": (i32, [P, P, P, P]),
            "h3d_batch_tune": (i32, [P, P, P, P, C.POINTER(i32)]),
            "h3d_batch_configure": (i32, [P, i32, i32, i32, i32, i32]),
            "h3d_batch_info": (i32, [P, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
            "h3d_batch_queue": (i32, [i32, P, P, P, P, i32, i32, i32, P, C.c_int64, C.POINTER(C.c_int64)]),
            "h3d_batch_set_wait_limit": (i32, [P, i64]),
            "h3d_batch_groups": (i32, [P, P, P]),
            "h3d_batch_get_queue": (i32, [P, P, i64, C.POINTER(i64)]),
            "h3d_batch_set_queue": (i32, [P, P, i64]),
            "h3d_batch_free": (i32, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _np(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


class H3DMatrix:
    """A built HODLR3D operator.  ``points``: (N, 3) float64 CUDA tensor.

    ``storage``: "factors" (the ACA factors of every ordered block, Alg. 1),
    "skeleton" (pivots and the LU of K(sigma,tau), entries recomputed in every
    product) or "symmetric" (each unordered pair compressed once, the mirror its
    transpose: an exactly symmetric operator with fewer stored bytes); see
    h3d_storage in include/h3d.h."""

    def __init__(self, points, kernel: str = "laplace", leaf_size: int = 128, tol: float = 1e-7,
                 precision: str = "fp32_3xtf32", rank_cap: int = 512, kappa: float = 1.0, lo=(-1.0, -1.0, -1.0),
                 side: float = 2.0, workspace_bytes: int = 0, admissibility: str = "hodlr3d",
                 storage: str = "factors", stream=None):
        import torch
        if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float64
                and points.dim() == 2 and points.shape[1] == 3):
            raise ValueError("points must be an (N, 3) float64 CUDA tensor")
        pts = points.contiguous()
        opt = Options()
        lib().h3d_default_options(C.byref(opt))
        opt.precision = PRECISIONS[precision]
        opt.kappa = kappa
        opt.rank_cap = rank_cap
        for d in range(3):
            opt.lo[d] = lo[d]
        opt.side = side
        opt.workspace_bytes = workspace_bytes
        opt.admissibility = ADMISSIBILITY[admissibility]
        opt.storage = STORAGE[storage]
        h = C.c_void_p()
        st = lib().h3d_build(pts.data_ptr(), pts.shape[0], KERNELS[kernel], leaf_size, tol, C.byref(opt),
                             _stream_ptr(stream), C.byref(h))
        if st != 0:
            raise H3DError(st, "h3d_build")
        self._h = h
        self.points = points            # the coordinates the operator currently holds
        self.N = pts.shape[0]
        self.precision = precision
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.kernel, self.leaf_size, self.tol = kernel, leaf_size, tol

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.h3d_free(self._h)
            self._h = None

    def _check_x(self, x):
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == self.dtype):
            raise ValueError(f"x must be a CUDA {self.dtype} tensor")
        if x.shape[0] != self.N or x.dim() not in (1, 2):
            raise ValueError("x must have N rows")

    def _apply(self, fn, x, out, stream):
        import torch
        self._check_x(x)
        nrhs = 1 if x.dim() == 1 else x.shape[1]
        # column-major N x nrhs == row-major nrhs x N
        xc = x.contiguous() if x.dim() == 1 else x.t().contiguous()
        if out is None:
            out = torch.empty_like(xc)
        st = fn(self._h, xc.data_ptr(), out.data_ptr(), nrhs, _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, fn.__name__)
        return out if x.dim() == 1 else out.t()

    def matvec(self, x, out=None, stream=None):
        """y = A~ x (Alg. 2).  x: (N,) or (N, nrhs) CUDA tensor of the handle's dtype."""
        return self._apply(lib().h3d_matvec, x, out, stream)

    def matvec_T(self, x, out=None, stream=None):
        """y = A~^T x."""
        return self._apply(lib().h3d_matvec_T, x, out, stream)

    def energy(self, q, grad: bool = True, stream=None):
        """E = 1/2 q^T A~ q (FP64, a 0-d CUDA tensor) and, if grad, dE/dq = 1/2 (A~ + A~^T) q."""
        import torch
        self._check_x(q)
        if q.dim() != 1:
            raise ValueError("q must be one column")
        qc = q.contiguous()
        E = torch.empty((), dtype=torch.float64, device=q.device)
        g = torch.empty_like(qc) if grad else None
        st = lib().h3d_energy(self._h, qc.data_ptr(), E.data_ptr(), g.data_ptr() if grad else None,
                              _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, "h3d_energy")
        return (E, g) if grad else E

    def forces(self, q, stream=None):
        """E (0-d FP64 CUDA tensor) and the forces F = -dE/dp (N x 3 FP64) for charges q,
        with the ACA pivots frozen (cross form of the admissible blocks)."""
        import torch
        self._check_x(q)
        if q.dim() != 1:
            raise ValueError("q must be one column")
        qc = q.contiguous()
        E = torch.empty((), dtype=torch.float64, device=q.device)
        F = torch.empty((self.N, 3), dtype=torch.float64, device=q.device)
        st = lib().h3d_forces(self._h, qc.data_ptr(), E.data_ptr(), F.data_ptr(), _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, "h3d_forces")
        return E, F

    def import_pivots(self, rank, sigma, tau, stream=None):
        """Re-form the operator from the given ACA pivots (format of export_pivots):
        same tree and lists, the factors formed from these pivots."""
        r = np.ascontiguousarray(rank, np.int32)
        sg = np.ascontiguousarray(sigma, np.int32)
        ta = np.ascontiguousarray(tau, np.int32)
        if sg.size != int(r.sum()) or ta.size != sg.size:
            raise ValueError("pivot arrays do not match the ranks")
        st = lib().h3d_import_pivots(self._h, _np(r), _np(sg) if sg.size else None, _np(ta) if ta.size else None,
                                     _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, "h3d_import_pivots")

    def set_points(self, points, stream=None):
        """Move the points (N x 3 float64 CUDA tensor, the caller's order), keeping
        the tree, lists and pivots; the factors are re-formed at the new positions.
        Costs one comparison pass when the coordinates are unchanged."""
        import torch
        if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float64
                and tuple(points.shape) == (self.N, 3)):
            raise ValueError("points must be an (N, 3) float64 CUDA tensor")
        pts = points.detach().contiguous()
        st = lib().h3d_set_points(self._h, pts.data_ptr(), _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, "h3d_set_points")
        self.points = points

    def matvec_raw(self, x_ptr: int, y_ptr: int, nrhs: int, stream=None, transpose: bool = False):
        """Call the C ABI directly on device pointers (column-major N x nrhs)."""
        fn = lib().h3d_matvec_T if transpose else lib().h3d_matvec
        st = fn(self._h, x_ptr, y_ptr, nrhs, _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, "h3d_matvec")

    def matvec_profile(self, x_ptr: int, y_ptr: int, nrhs: int, stream=None) -> list[float]:
        """One product with per-phase CUDA-event timing (ms): permute, gather, reduce, leaf."""
        ms = (C.c_float * 4)()
        st = lib().h3d_matvec_profile(self._h, x_ptr, y_ptr, nrhs, _stream_ptr(stream), ms, 4)
        if st != 0:
            raise H3DError(st, "h3d_matvec_profile")
        return list(ms)

    def matvec_host(self, x: np.ndarray, y: np.ndarray | None = None, stream=None) -> np.ndarray:
        """y = A~ x with host arrays (x: (N,) or column-major (N, nrhs))."""
        dt = np.float64 if self.precision == "fp64" else np.float32
        if x.dtype != dt or x.shape[0] != self.N:
            raise ValueError(f"x must be a host {dt.__name__} array with N rows")
        nrhs = 1 if x.ndim == 1 else x.shape[1]
        if not (x.flags.f_contiguous or x.ndim == 1):
            raise ValueError("x must be column-major")
        if y is None:
            y = np.empty_like(x, order="F")
        st = lib().h3d_matvec_host(self._h, _np(x), _np(y), nrhs, _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, "h3d_matvec_host")
        return y

    def matvec_host_ptr(self, x_ptr: int, y_ptr: int, nrhs: int, stream=None):
        st = lib().h3d_matvec_host(self._h, x_ptr, y_ptr, nrhs, _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, "h3d_matvec_host")

    def stats(self) -> dict:
        s = Stats()
        st = lib().h3d_get_stats(self._h, C.byref(s))
        if st != 0:
            raise H3DError(st, "h3d_get_stats")
        return s.as_dict()

    def export_tree(self) -> dict:
        s = self.stats()
        N, nb, L = s["N"], s["n_boxes"], s["depth"]
        perm = np.zeros(N, np.int64)
        keys = np.zeros(N, np.uint64)
        nbox = np.zeros(L + 1, np.int32)
        bkey = np.zeros(nb, np.uint64)
        bs = np.zeros(nb, np.int64)
        be = np.zeros(nb, np.int64)
        st = lib().h3d_export_tree(self._h, _np(perm), _np(keys), _np(nbox), _np(bkey), _np(bs), _np(be))
        if st != 0:
            raise H3DError(st, "h3d_export_tree")
        return {"L": L, "perm": perm, "keys": keys, "nbox": nbox, "box_key": bkey, "box_start": bs, "box_end": be}

    def export_lists(self) -> dict:
        s = self.stats()
        nb, nn = s["n_blocks"], s["n_near"]
        a = {k: np.zeros(max(nb, 1), np.int32) for k in ("level", "tgt", "src", "cls")}
        b = {k: np.zeros(max(nn, 1), np.int32) for k in ("near_tgt", "near_src", "near_cls")}
        st = lib().h3d_export_lists(self._h, _np(a["level"]), _np(a["tgt"]), _np(a["src"]), _np(a["cls"]),
                                    _np(b["near_tgt"]), _np(b["near_src"]), _np(b["near_cls"]))
        if st != 0:
            raise H3DError(st, "h3d_export_lists")
        out = {k: v[:nb] for k, v in a.items()}
        out.update({k: v[:nn] for k, v in b.items()})
        return out

    def export_pivots(self) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        s = self.stats()
        rank = np.zeros(max(s["n_blocks"], 1), np.int32)
        sig = np.zeros(max(s["sum_rank"], 1), np.int32)
        tau = np.zeros(max(s["sum_rank"], 1), np.int32)
        st = lib().h3d_export_pivots(self._h, _np(rank), _np(sig), _np(tau))
        if st != 0:
            raise H3DError(st, "h3d_export_pivots")
        return rank[:s["n_blocks"]], sig[:s["sum_rank"]], tau[:s["sum_rank"]]


def debug_fail_alloc(after: int):
    """Test hook: the next `after` device allocations of the library succeed and the
    one after them fails (H3D_ERR_OOM); a negative value switches it off."""
    lib().h3d_debug_fail_alloc(int(after))


def batch_queue(n_points, n_gather, n_split, n_leaves, near_group=4, leaf_group=2, lag=0) -> np.ndarray:
    """The persistent batch form's work queue for operators of these sizes
    (h3d_batch_queue; host only): an (items x 4) int32 array of (operator,
    kind, first, count), kind 0 gather, 1 near field, 2 reduce, 3 leaf,
    4 permute."""
    n = len(n_points)
    npts = np.ascontiguousarray(n_points, np.int64)
    ng, ns, nl = (np.ascontiguousarray(v, np.int32) for v in (n_gather, n_split, n_leaves))
    cnt = C.c_int64()
    st = lib().h3d_batch_queue(n, _np(npts), _np(ng), _np(ns), _np(nl), near_group, leaf_group, lag, None, 0,
                               C.byref(cnt))
    if st != 0:
        raise H3DError(st, "h3d_batch_queue")
    out = np.zeros((max(cnt.value, 1), 4), np.int32)
    st = lib().h3d_batch_queue(n, _np(npts), _np(ng), _np(ns), _np(nl), near_group, leaf_group, lag, _np(out),
                               cnt.value, C.byref(cnt))
    if st != 0:
        raise H3DError(st, "h3d_batch_queue")
    return out[:cnt.value]


class H3DBatch:
    """Products of several H3DMatrix operators (independent point clouds), one
    column each, as one persistent launch (all FP32 or all FP64 factor-storage
    matrices) or as one CUDA graph of every matrix's own kernels (h3d_batch_*).
    The matrices must outlive the batch."""

    def __init__(self, mats):
        self.mats = list(mats)
        arr = (C.c_void_p * len(self.mats))(*[m._h for m in self.mats])
        h = C.c_void_p()
        st = lib().h3d_batch_create(arr, len(self.mats), C.byref(h))
        if st != 0:
            raise H3DError(st, "h3d_batch_create")
        self._b = h

    def _ptrs(self, xs, ys):
        for m, x, y in zip(self.mats, xs, ys):
            m._check_x(x)
            m._check_x(y)
            if x.dim() != 1 or y.dim() != 1 or not x.is_contiguous() or not y.is_contiguous():
                raise ValueError("one contiguous column per cloud")
        n = len(self.mats)
        return (C.c_void_p * n)(*[x.data_ptr() for x in xs]), (C.c_void_p * n)(*[y.data_ptr() for y in ys])

    def matvec(self, xs, ys, stream=None):
        """ys[i] = A_i xs[i] for every cloud (device tensors, kept by the caller)."""
        xp, yp = self._ptrs(xs, ys)
        st = lib().h3d_batch_matvec(self._b, xp, yp, _stream_ptr(stream))
        if st != 0:
            raise H3DError(st, "h3d_batch_matvec")

    def tune(self, xs, ys, stream=None) -> int:
        """Time both forms and keep the fastest; returns the graph's branch count,
        or 0 when the persistent form won."""
        xp, yp = self._ptrs(xs, ys)
        nb = C.c_int()
        st = lib().h3d_batch_tune(self._b, xp, yp, _stream_ptr(stream), C.byref(nb))
        if st != 0:
            raise H3DError(st, "h3d_batch_tune")
        return nb.value

    def set_mode(self, persistent: bool, ctas_per_sm: int = 0, near_group: int = 0, leaf_group: int = 0,
                 lag: int = -1):
        """Select the persistent kernel or the graph form, and the persistent
        form's CTAs per SM, leaves per near / leaf item and queue lag (0, or -1
        for lag: keep the current value)."""
        st = lib().h3d_batch_configure(self._b, 1 if persistent else 0, int(ctas_per_sm), int(near_group),
                                       int(leaf_group), int(lag))
        if st != 0:
            raise H3DError(st, "h3d_batch_configure")

    def info(self) -> dict:
        """{"persistent": 1 | 0 | -1 (unavailable), "ctas_per_sm": .., "branches": ..}"""
        p, c, b = C.c_int(), C.c_int(), C.c_int()
        st = lib().h3d_batch_info(self._b, C.byref(p), C.byref(c), C.byref(b))
        if st != 0:
            raise H3DError(st, "h3d_batch_info")
        return {"persistent": p.value, "ctas_per_sm": c.value, "branches": b.value}

    def groups(self) -> tuple[np.ndarray, np.ndarray]:
        """The persistent form's leaves per near-field item and per leaf item, per matrix."""
        n = len(self.mats)
        ng, lg = np.zeros(n, np.int32), np.zeros(n, np.int32)
        st = lib().h3d_batch_groups(self._b, _np(ng), _np(lg))
        if st != 0:
            raise H3DError(st, "h3d_batch_groups")
        return ng, lg

    def set_wait_limit(self, ns: int):
        """Bound of every wait of the persistent kernel, in nanoseconds."""
        st = lib().h3d_batch_set_wait_limit(self._b, int(ns))
        if st != 0:
            raise H3DError(st, "h3d_batch_set_wait_limit")

    def queue(self) -> np.ndarray:
        """The persistent form's work queue, (items x 4) int32: (operator, kind, first, count)."""
        cnt = C.c_int64()
        st = lib().h3d_batch_get_queue(self._b, None, 0, C.byref(cnt))
        if st != 0:
            raise H3DError(st, "h3d_batch_get_queue")
        out = np.zeros((max(cnt.value, 1), 4), np.int32)
        st = lib().h3d_batch_get_queue(self._b, _np(out), cnt.value, C.byref(cnt))
        if st != 0:
            raise H3DError(st, "h3d_batch_get_queue")
        return out[:cnt.value]

    def set_queue(self, items=None):
        """Run the persistent kernel on these items ((k x 4) int32), or, with None,
        on the queue of the current settings."""
        if items is None:
            st = lib().h3d_batch_set_queue(self._b, None, 0)
        else:
            it = np.ascontiguousarray(items, np.int32).reshape(-1, 4)
            st = lib().h3d_batch_set_queue(self._b, _np(it), it.shape[0])
        if st != 0:
            raise H3DError(st, "h3d_batch_set_queue")

    def free(self):
        if getattr(self, "_b", None) is not None and _lib is not None:
            _lib.h3d_batch_free(self._b)
            self._b = None

    def __del__(self):
        self.free()
