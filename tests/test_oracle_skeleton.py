"""Pins for the oracle's skeleton-form product (pivots + K(sigma,tau) only).

* With the same pivots it equals the ACA-factor product up to rounding times the
  condition of K(sigma,tau) (ACA's factors are that cross form, Sec. 4.1).
* Full rank (tol = 0): it equals the dense direct sum.
* Its error against the direct sum tracks the ACA tolerance like the product's.
"""
import numpy as np

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_skeleton_equals_aca_product():
    p = I.uniform(3000, 261)
    o = O.Oracle(p, leaf_size=32, tol=1e-6).compress()
    x = I.rhs_normal(3000, 1, 262)[:, 0]
    assert rel(o.matvec_skeleton(x), o.matvec(x)) <= 1e-9


def test_skeleton_full_rank_is_dense():
    p = I.uniform(600, 263)
    o = O.Oracle(p, leaf_size=10, tol=0.0).compress()
    x = I.rhs_uniform(600, 1, 264)[:, 0]
    assert rel(o.matvec_skeleton(x), O.direct(p, x)) <= 1e-12


def test_skeleton_error_tracks_tolerance():
    p = I.uniform(4000, 265)
    x = I.rhs_uniform(4000, 1, 266)[:, 0]
    y = O.direct(p, x)
    e = [rel(O.Oracle(p, leaf_size=40, tol=t).compress().matvec_skeleton(x), y) for t in (1e-4, 1e-6, 1e-8)]
    assert e[0] > e[1] > e[2] and e[2] < 1e-6


def test_skeleton_transpose_is_exact_transpose():
    p = I.uniform(500, 267)
    o = O.Oracle(p, leaf_size=10, tol=1e-5).compress()
    E = np.eye(500)
    A = np.stack([o.matvec_skeleton(E[:, j]) for j in range(500)], axis=1)
    AT = np.stack([o.matvec_skeleton(E[:, j], transpose=True) for j in range(500)], axis=1)
    assert np.abs(AT - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.norm(A - A.T) > 0
