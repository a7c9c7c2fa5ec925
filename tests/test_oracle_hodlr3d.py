"""Pins for the oracle's HODLR3D product (Alg. 2) against the dense sum O1.

* Depth 0 (one leaf) is the dense product: equal to O1 to rounding.
* Full-rank compression (tol = 0) on deeper trees equals O1 to rounding.
* The error falls with the ACA tolerance and sits near the paper's figures.
* The transpose product is the exact transpose of the forward operator.
* The forward operator is symmetric up to the tolerance (K = K^T).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_depth_zero_equals_dense():
    p = I.grid(8)
    x = I.rhs_uniform(512, 2, 0)
    o = O.Oracle(p, leaf_size=512).compress()
    assert o.L == 0 and o.n_blocks == 0
    assert rel(o.matvec(x), O.direct(p, x)) <= 1e-14


@pytest.mark.parametrize("pts,leaf", [(I.grid(8), 64), (I.grid(8), 8), (I.uniform(1200, 61), 20)])
def test_full_rank_equals_dense(pts, leaf):
    o = O.Oracle(pts, leaf_size=leaf, tol=0.0).compress()
    assert o.L >= 1
    x = I.rhs_normal(pts.shape[0], 1, 62)[:, 0]
    assert rel(o.matvec(x), O.direct(pts, x)) <= 1e-12


def test_error_tracks_tolerance():
    p = I.uniform(6000, 63)
    x = I.rhs_uniform(6000, 1, 64)[:, 0]
    y = O.direct(p, x)
    errs = []
    for tol in (1e-3, 1e-5, 1e-7, 1e-9):
        o = O.Oracle(p, leaf_size=48, tol=tol).compress()
        errs.append(rel(o.matvec(x), y))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    for tol, e in zip((1e-3, 1e-5, 1e-7, 1e-9), errs):
        assert 1e-3 * tol < e < 10 * tol


def test_error_near_paper_figure():
    # Fig. oneOverR_2, HODLR3D at eps = 1e-7: relative errors 1.7e-8 .. 7.2e-8
    # for N = 8000 .. 1e6 (order of magnitude only; different leaf and ACA).
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "paper_hodlr3d_1overr_eps1e-7.txt"))
            if ln.strip() and not ln.startswith("#")]
    paper = {int(r[0]): float(r[1]) for r in rows[1:]}
    N = 8000
    p = I.uniform(N, 65)
    x = I.rhs_uniform(N, 1, 66)[:, 0]
    o = O.Oracle(p, leaf_size=64, tol=1e-7).compress()
    e = rel(o.matvec(x), O.direct(p, x))
    assert paper[8000] / 30 < e < paper[8000] * 30


def test_transpose_is_exact_transpose():
    p = I.uniform(700, 67)
    o = O.Oracle(p, leaf_size=12, tol=1e-5).compress()
    E = np.eye(700)
    A = o.matvec(E)
    AT = o.matvec(E, transpose=True)
    assert np.abs(AT - A.T).max() <= 1e-13 * np.abs(A).max()
    # and the operator is symmetric up to the ACA tolerance
    assert np.linalg.norm(A - A.T) / np.linalg.norm(A) < 1e-4
    assert np.linalg.norm(A - A.T) > 0  # ordered compression: not exactly symmetric


def test_multiple_rhs_columns_independent():
    p = I.uniform(1000, 68)
    o = O.Oracle(p, leaf_size=16, tol=1e-6).compress()
    X = I.rhs_normal(1000, 3, 69)
    Y = o.matvec(X)
    for c in range(3):
        assert np.array_equal(Y[:, c], o.matvec(X[:, c]))


@pytest.mark.parametrize("mode", ["strong", "weak"])
def test_variants_full_rank_equal_dense_and_track_tol(mode):
    p = I.uniform(2500, 71)
    x = I.rhs_uniform(2500, 1, 72)[:, 0]
    y = O.direct(p, x)
    o = O.Oracle(p, leaf_size=24, tol=0.0, admissibility=mode).compress()
    assert rel(o.matvec(x), y) <= 1e-12
    e5 = rel(O.Oracle(p, leaf_size=24, tol=1e-5, admissibility=mode).compress().matvec(x), y)
    e8 = rel(O.Oracle(p, leaf_size=24, tol=1e-8, admissibility=mode).compress().matvec(x), y)
    assert e8 < e5 < 1e-3


def test_rank_ordering_of_formats():
    # the paper's Figs. oneOverR_2 etc.: HODLR's maximum rank exceeds HODLR3D's,
    # which exceeds the strong-admissibility H-matrix's
    p = I.uniform(8000, 73)
    mx = {m: O.Oracle(p, leaf_size=32, tol=1e-7, admissibility=m).compress().pivots()[0].max()
          for m in ("weak", "hodlr3d", "strong")}
    assert mx["weak"] > mx["hodlr3d"] > mx["strong"]
