"""CPU FP64 oracle for the HODLR3D matrix-vector product -- TEST INFRASTRUCTURE.

This module wraps ``h3d_oracle.c`` (plain C, FP64) with ctypes.  It is the
reference the CUDA library is checked against and is used only by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.  It imports
nothing from the CUDA package and the CUDA package imports nothing from it.

Functions and the passage of arXiv 2307.16303 each one follows:

* :func:`direct`, :func:`direct_rows` -- O1, the dense sum of Eq. (Laplace3D):
  y_i = sum_{j != i} f(|r_i - r_j|) x_j.
* :func:`direct_forces_rows` -- the gradient of O1's energy q^T K q / 2 in the
  point positions (exact forces on selected points).
* :func:`morton` -- Sec. 2.1 recursive subdivision of B = [-1, 1]^3.
* :class:`Oracle` -- Alg. 1 (tree, interaction lists, ACA pivots, Sec. 4.1
  Eq. prank) and Alg. 2 (matrix-vector product and its transpose); the energy
  q^T K~ q / 2 and its gradient in the point positions with the pivots frozen
  (the cross form of Eq. prank differentiated entry by entry); with
  ``admissibility="strong"`` / ``"weak"`` the paper's comparison formats on the
  same octree (H-matrix with eta = sqrt(3), Eq. adm; HODLR, Sec. 2.3); with
  ``symmetric=True`` each unordered admissible pair compressed once, its
  mirror block taking the transposed factors (K symmetric, Eq. prank
  transposed).

Pins (tests under ``tests/`` marked ``not gpu``) fix each function against
something other than itself: closed-form potentials of symmetric point sets,
the symmetry of K, the depth-0 tree reducing to the dense sum, full-rank ACA
reproducing the block, the skeleton identity of Eq. prank checked with a dense
solve, exact block counts derived by hand and by geometric brute force, the
coverage of the N x N matrix by exactly one block per entry, the error falling
with the ACA tolerance, and the rank growth by interaction class of Table
"rankgrowth", and, for symmetric storage, the product being an exactly
symmetric matrix whose primary blocks carry the pivots of the ordered mode.
No function here is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h3d_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libh3d_oracle.so")

KERNELS = {"laplace": 0, "yukawa": 1, "inv_r4": 2, "cos_r": 3}
ADMISSIBILITY = {"hodlr3d": 0, "strong": 1, "weak": 2}
STATUS = {0: "ok", 1: "bad argument", 2: "point outside the domain", 3: "out of memory",
          5: "ACA rank cap reached", 8: "tree deeper than 21 levels"}
CLS_NAMES = {0: "self", 1: "face", 2: "edge", 3: "vertex", 4: "far"}


def direct_forces_rows(points, q, rows, kernel: str = "laplace", kappa: float = 1.0) -> np.ndarray:
    """Exact forces -dE/dp_i of the dense energy q^T K q / 2 on the given points (O1's gradient)."""
    p = np.ascontiguousarray(points, np.float64)
    qf = np.ascontiguousarray(q, np.float64).reshape(p.shape[0])
    r = np.ascontiguousarray(rows, np.int64)
    out = np.zeros((r.shape[0], 3), np.float64)
    _check(_load().h3do_direct_forces_rows(KERNELS[kernel], kappa, _ptr(p), p.shape[0], _ptr(qf), _ptr(r),
                                           r.shape[0], _ptr(out)))
    return out


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle status {status}: {STATUS.get(status, '?')}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so fma() is the only FMA)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        i64, i32, f64 = C.c_int64, C.c_int, C.c_double
        sig = {
            "h3do_kernel": (f64, [i32, f64, P, P]),
            "h3do_direct": (i32, [i32, f64, P, i64, P, i32, P]),
            "h3do_direct_rows": (i32, [i32, f64, P, i64, P, i32, P, i64, P]),
            "h3do_num_threads": (i32, []),
            "h3do_morton": (i32, [P, i64, P, f64, P]),
            "h3do_create": (P, [P, i64, i32, f64, i32, f64, i32, P, f64, C.POINTER(C.c_int)]),
            "h3do_create_adm": (P, [P, i64, i32, f64, i32, f64, i32, P, f64, i32, C.POINTER(C.c_int)]),
            "h3do_free": (None, [P]),
            "h3do_depth": (i32, [P]),
            "h3do_num_blocks": (i64, [P]),
            "h3do_num_near": (i64, [P]),
            "h3do_num_boxes": (i64, [P]),
            "h3do_export_tree": (None, [P, P, P, P, P, P, P]),
            "h3do_export_lists": (None, [P, P, P, P, P, P, P, P]),
            "h3do_compress": (i32, [P]),
            "h3do_set_symmetric": (i32, [P, i32]),
            "h3do_num_pivots": (i64, [P]),
            "h3do_get_pivots": (i32, [P, P, P, P]),
            "h3do_set_pivots": (i32, [P, P, P, P]),
            "h3do_block_factors": (i32, [P, i64, P, P]),
            "h3do_block_geometry": (i32, [P, i64, C.POINTER(i64), C.POINTER(C.c_int),
                                          C.POINTER(i64), C.POINTER(C.c_int)]),
            "h3do_apply": (i32, [P, P, i32, P, i32]),
            "h3do_energy_forces": (i32, [P, P, P, P]),
            "h3do_apply_skeleton": (i32, [P, P, P, i32]),
            "h3do_direct_forces_rows": (i32, [i32, f64, P, i64, P, P, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(st: int):
    if st != 0:
        raise OracleError(st)


def num_threads() -> int:
    return int(_load().h3do_num_threads())


def kernel_value(kind: str, a, b, kappa: float = 1.0) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(_load().h3do_kernel(KERNELS[kind], kappa, _ptr(a), _ptr(b)))


def _as_x(x: np.ndarray, n: int) -> tuple[np.ndarray, int, bool]:
    x = np.asarray(x, dtype=np.float64)
    vec = x.ndim == 1
    if vec:
        x = x[:, None]
    if x.shape[0] != n:
        raise ValueError("x must have N rows")
    return np.asfortranarray(x), x.shape[1], vec


def direct(points: np.ndarray, x: np.ndarray, kernel: str = "laplace", kappa: float = 1.0) -> np.ndarray:
    """O1: y = K x with K(i,i) = 0 (Eq. Laplace3D), FP64, compensated sums."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[0]
    xf, nrhs, vec = _as_x(x, n)
    y = np.zeros((n, nrhs), dtype=np.float64, order="F")
    _check(_load().h3do_direct(KERNELS[kernel], kappa, _ptr(pts), n, _ptr(xf), nrhs, _ptr(y)))
    return y[:, 0] if vec else y


def direct_rows(points: np.ndarray, x: np.ndarray, rows: np.ndarray, kernel: str = "laplace",
                kappa: float = 1.0) -> np.ndarray:
    """O1 on selected rows only: returns (K x)[rows]."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[0]
    xf, nrhs, vec = _as_x(x, n)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.zeros((rows.size, nrhs), dtype=np.float64, order="F")
    _check(_load().h3do_direct_rows(KERNELS[kernel], kappa, _ptr(pts), n, _ptr(xf), nrhs,
                                    _ptr(rows), rows.size, _ptr(y)))
    return y[:, 0] if vec else y


def morton(points: np.ndarray, lo=(-1.0, -1.0, -1.0), side: float = 2.0) -> np.ndarray:
    pts = np.ascontiguousarray(points, dtype=np.float64)
    keys = np.zeros(pts.shape[0], dtype=np.uint64)
    lo_a = np.ascontiguousarray(lo, dtype=np.float64)
    _check(_load().h3do_morton(_ptr(pts), pts.shape[0], _ptr(lo_a), side, _ptr(keys)))
    return keys


class Oracle:
    """Alg. 1 + Alg. 2 on the CPU in FP64.

    ``Oracle(points, ...)`` forms the tree and the lists; :meth:`compress` runs
    ACA on every admissible block and keeps the pivots (the paper's storage,
    Sec. 4.1); :meth:`set_pivots` freezes pivots found elsewhere; :meth:`matvec`
    applies Alg. 2, re-forming each block's factors from the pivots.
    """

    def __init__(self, points, kernel: str = "laplace", leaf_size: int = 64, tol: float = 1e-7,
                 rank_cap: int = 512, kappa: float = 1.0, lo=(-1.0, -1.0, -1.0), side: float = 2.0,
                 admissibility: str = "hodlr3d", symmetric: bool = False):
        lib = _load()
        self.points = np.ascontiguousarray(points, dtype=np.float64)
        self.N = self.points.shape[0]
        lo_a = np.ascontiguousarray(lo, dtype=np.float64)
        st = C.c_int(0)
        self._h = lib.h3do_create_adm(_ptr(self.points), self.N, KERNELS[kernel], kappa, leaf_size, tol,
                                      rank_cap, _ptr(lo_a), side, ADMISSIBILITY[admissibility], C.byref(st))
        if not self._h:
            raise OracleError(st.value)
        self.kernel, self.kappa, self.leaf_size, self.tol = kernel, kappa, leaf_size, tol
        self.admissibility = admissibility
        self.L = lib.h3do_depth(self._h)
        self.n_blocks = lib.h3do_num_blocks(self._h)
        self.n_near = lib.h3do_num_near(self._h)
        self.symmetric = bool(symmetric)
        if symmetric:
            _check(lib.h3do_set_symmetric(self._h, 1))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.h3do_free(self._h)
            self._h = None

    # --- tree and lists -------------------------------------------------
    def tree(self) -> dict:
        lib = _load()
        nb = lib.h3do_num_boxes(self._h)
        perm = np.zeros(self.N, np.int64)
        keys = np.zeros(self.N, np.uint64)
        nbox = np.zeros(self.L + 1, np.int32)
        bkey = np.zeros(nb, np.uint64)
        bs = np.zeros(nb, np.int64)
        be = np.zeros(nb, np.int64)
        lib.h3do_export_tree(self._h, _ptr(perm), _ptr(keys), _ptr(nbox), _ptr(bkey), _ptr(bs), _ptr(be))
        return {"L": self.L, "perm": perm, "keys": keys, "nbox": nbox, "box_key": bkey,
                "box_start": bs, "box_end": be}

    def lists(self) -> dict:
        nb, nn = self.n_blocks, self.n_near
        a = {k: np.zeros(nb, np.int32) for k in ("level", "tgt", "src", "cls")}
        b = {k: np.zeros(nn, np.int32) for k in ("near_tgt", "near_src", "near_cls")}
        _load().h3do_export_lists(self._h, _ptr(a["level"]), _ptr(a["tgt"]), _ptr(a["src"]), _ptr(a["cls"]),
                                  _ptr(b["near_tgt"]), _ptr(b["near_src"]), _ptr(b["near_cls"]))
        a.update(b)
        return a

    def block_geometry(self, b: int) -> tuple[int, int, int, int]:
        xs, ys = C.c_int64(0), C.c_int64(0)
        m, n = C.c_int(0), C.c_int(0)
        _check(_load().h3do_block_geometry(self._h, b, C.byref(xs), C.byref(m), C.byref(ys), C.byref(n)))
        return xs.value, m.value, ys.value, n.value

    # --- compression ----------------------------------------------------
    def compress(self) -> "Oracle":
        _check(_load().h3do_compress(self._h))
        return self

    def pivots(self) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        lib = _load()
        tot = lib.h3do_num_pivots(self._h)
        if tot < 0:
            raise OracleError(1)
        rank = np.zeros(self.n_blocks, np.int32)
        sig = np.zeros(max(tot, 1), np.int32)
        tau = np.zeros(max(tot, 1), np.int32)
        _check(lib.h3do_get_pivots(self._h, _ptr(rank), _ptr(sig), _ptr(tau)))
        return rank, sig[:tot], tau[:tot]

    def set_pivots(self, rank, sigma, tau) -> "Oracle":
        rank = np.ascontiguousarray(rank, dtype=np.int32)
        sigma = np.ascontiguousarray(sigma, dtype=np.int32)
        tau = np.ascontiguousarray(tau, dtype=np.int32)
        if rank.size != self.n_blocks or sigma.size != int(rank.sum()) or tau.size != sigma.size:
            raise ValueError("pivot arrays do not match the block list")
        _check(_load().h3do_set_pivots(self._h, _ptr(rank), _ptr(sigma), _ptr(tau)))
        return self

    def block_factors(self, b: int) -> tuple[np.ndarray, np.ndarray]:
        """U (m x r) and V (n x r) of block b, formed from the stored pivots."""
        rank, _, _ = self.pivots()
        _, m, _, n = self.block_geometry(b)
        r = int(rank[b])
        U = np.zeros((m, max(r, 1)), np.float64, order="F")
        V = np.zeros((n, max(r, 1)), np.float64, order="F")
        _check(_load().h3do_block_factors(self._h, b, _ptr(U), _ptr(V)))
        return U[:, :r], V[:, :r]

    # --- Alg. 2 ---------------------------------------------------------
    def matvec(self, x, transpose: bool = False) -> np.ndarray:
        xf, nrhs, vec = _as_x(x, self.N)
        y = np.zeros((self.N, nrhs), np.float64, order="F")
        _check(_load().h3do_apply(self._h, _ptr(xf), nrhs, _ptr(y), 1 if transpose else 0))
        return y[:, 0] if vec else y

    def matvec_skeleton(self, x, transpose: bool = False) -> np.ndarray:
        """The product in the skeleton form the paper stores (Sec. 4.1): near blocks
        plus K(X,tau) K(sigma,tau)^{-1} K(sigma,Y) x_Y per admissible block (or the
        transposed operator)."""
        xf = np.ascontiguousarray(x, np.float64).reshape(self.N)
        y = np.zeros(self.N, np.float64)
        _check(_load().h3do_apply_skeleton(self._h, _ptr(xf), _ptr(y), 1 if transpose else 0))
        return y

    # --- forces: gradient of E = q^T K~ q / 2 in the point positions -------
    def energy_forces(self, q) -> tuple[float, np.ndarray]:
        """E and dE/dp (N x 3, the caller's order) with the pivots frozen: near
        blocks exact, admissible blocks in the cross form K(X,tau) K(sigma,tau)^{-1}
        K(sigma,Y) of Eq. prank, every kernel entry differentiated."""
        qf = np.ascontiguousarray(q, np.float64).reshape(self.N)
        E = np.zeros(1, np.float64)
        G = np.zeros((self.N, 3), np.float64)
        _check(_load().h3do_energy_forces(self._h, _ptr(qf), _ptr(E), _ptr(G)))
        return float(E[0]), G

    def sorted_points(self) -> np.ndarray:
        return self.points[self.tree()["perm"]]


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
