"""Pins for the energy E = 1/2 q^T A~ q and its gradient 1/2 (A~ + A~^T) q on the oracle.

* Central differences of E (computed with the forward product only) equal the
  gradient built from the forward and transpose products: E is quadratic in q,
  so the difference quotient is exact up to rounding for any step.
* Full rank (tol = 0): A~ is the dense symmetric matrix, so the gradient is A q
  from the direct sum.
"""
import numpy as np

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I


def energy(o, q):
    return 0.5 * float(q @ o.matvec(q))


def grad(o, q):
    return 0.5 * (o.matvec(q) + o.matvec(q, transpose=True))


def test_central_differences_match_gradient():
    p = I.uniform(900, 201)
    o = O.Oracle(p, leaf_size=16, tol=1e-4).compress()   # loose: A~ visibly non-symmetric
    q = I.rhs_uniform(900, 1, 202)[:, 0]
    g = grad(o, q)
    rng = np.random.default_rng(203)
    for i in rng.choice(900, 12, replace=False):
        for h in (1e-2, 1e-4):
            e = np.zeros(900)
            e[i] = h
            fd = (energy(o, q + e) - energy(o, q - e)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-9 * np.abs(g).max()
    # the gradient differs from the forward product alone (A~ != A~^T)
    assert np.abs(g - o.matvec(q)).max() > 1e-9 * np.abs(g).max()


def test_full_rank_gradient_is_dense_product():
    p = I.uniform(700, 204)
    o = O.Oracle(p, leaf_size=12, tol=0.0).compress()
    q = I.rhs_normal(700, 1, 205)[:, 0]
    dense = O.direct(p, q)
    g = grad(o, q)
    assert np.linalg.norm(g - dense) <= 1e-12 * np.linalg.norm(dense)
    assert abs(energy(o, q) - 0.5 * q @ dense) <= 1e-12 * abs(0.5 * q @ dense)
