"""Pins for the oracle's energy / position gradient (forces), pivots frozen.

* Two charges (depth 0, only the near block): E = q1 q2 f(d) and the gradient
  q1 q2 f'(d) (p1 - p2) / d, written out for the Laplace and Yukawa kernels.
* Translation invariance: with the pivots frozen the energy depends on point
  differences only, so the gradients sum to zero.
* Full rank (tol = 0): the energy and its gradient equal those of the dense
  direct sum, checked by central differences of O1's energy.
* Compressed (loose tolerance): central differences of the energy of the
  oracle's ACA product, rebuilt at moved points with the same frozen pivots and
  the same tree, match the gradient (an independent code path: the product
  forms U, V by the ACA recursion, the gradient uses the cross form).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I

FOUR_PI = 4 * np.pi


@pytest.mark.parametrize("kern,kappa", [("laplace", 1.0), ("yukawa", 0.7)])
def test_two_charges_closed_form(kern, kappa):
    p = np.array([[0.1, -0.2, 0.3], [-0.25, 0.4, 0.05]])
    q = np.array([0.8, -1.3])
    o = O.Oracle(p, leaf_size=4, kernel=kern, kappa=kappa).compress()
    E, G = o.energy_forces(q)
    dvec = p[0] - p[1]
    d = np.linalg.norm(dvec)
    if kern == "laplace":
        f, fp = 1 / (FOUR_PI * d), -1 / (FOUR_PI * d * d)
    else:
        f = np.exp(-kappa * d) / (FOUR_PI * d)
        fp = -np.exp(-kappa * d) * (1 + kappa * d) / (FOUR_PI * d * d)
    assert abs(E - q[0] * q[1] * f) <= 1e-15 * abs(E)
    g1 = q[0] * q[1] * fp * dvec / d
    assert np.allclose(G[0], g1, rtol=1e-14, atol=0) and np.allclose(G[1], -g1, rtol=1e-14, atol=0)


def test_gradients_sum_to_zero():
    p = I.uniform(1500, 231)
    o = O.Oracle(p, leaf_size=20, tol=1e-6).compress()
    _, G = o.energy_forces(I.rhs_uniform(1500, 1, 232)[:, 0])
    assert np.abs(G.sum(axis=0)).max() <= 1e-12 * np.abs(G).sum()


def _dense_energy(p, q):
    return 0.5 * q @ O.direct(p, q)


def test_full_rank_equals_dense_by_central_differences():
    p = I.uniform(600, 233)
    q = I.rhs_uniform(600, 1, 234)[:, 0]
    o = O.Oracle(p, leaf_size=10, tol=0.0).compress()
    assert o.L >= 2
    E, G = o.energy_forces(q)
    assert abs(E - _dense_energy(p, q)) <= 1e-12 * abs(E)
    rng = np.random.default_rng(235)
    h = 1e-6
    for i in rng.choice(600, 6, replace=False):
        for d in range(3):
            pp, pm = p.copy(), p.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = (_dense_energy(pp, q) - _dense_energy(pm, q)) / (2 * h)
            assert abs(fd - G[i, d]) <= 1e-6 * np.abs(G[i]).max() + 1e-9


def test_compressed_gradient_by_central_differences():
    p = I.uniform(2000, 236)
    q = I.rhs_uniform(2000, 1, 237)[:, 0]
    kw = dict(leaf_size=24, tol=1e-4)
    o = O.Oracle(p, **kw).compress()
    piv = o.pivots()
    E, G = o.energy_forces(q)
    # the cross form and the ACA product agree to rounding (times cond K(sigma,tau))
    assert abs(E - 0.5 * q @ o.matvec(q)) <= 1e-9 * abs(E)
    t0 = o.tree()
    rng = np.random.default_rng(238)
    h = 1e-5
    checked = 0
    for i in rng.choice(2000, 20, replace=False):
        for d in range(3):
            Es = []
            for sgn in (1, -1):
                pm = p.copy()
                pm[i, d] += sgn * h
                om = O.Oracle(pm, **kw)
                tm = om.tree()
                if not (np.array_equal(tm["perm"], t0["perm"]) and np.array_equal(tm["box_start"], t0["box_start"])):
                    break
                om.set_pivots(*piv)
                Es.append(0.5 * q @ om.matvec(q))
            if len(Es) < 2:
                continue
            fd = (Es[0] - Es[1]) / (2 * h)
            assert abs(fd - G[i, d]) <= 1e-5 * np.abs(G[i]).max() + 1e-9
            checked += 1
    assert checked >= 30


@pytest.mark.parametrize("kern", ["laplace", "yukawa", "inv_r4", "cos_r"])
def test_direct_forces_by_central_differences(kern):
    p = I.uniform(300, 239)
    q = I.rhs_uniform(300, 1, 240)[:, 0]
    rows = np.array([0, 7, 123, 299])
    F = O.direct_forces_rows(p, q, rows, kernel=kern, kappa=0.9)
    h = 1e-6
    for r, i in enumerate(rows):
        for d in range(3):
            pp, pm = p.copy(), p.copy()
            pp[i, d] += h
            pm[i, d] -= h
            ep = 0.5 * q @ O.direct(pp, q, kernel=kern, kappa=0.9)
            em = 0.5 * q @ O.direct(pm, q, kernel=kern, kappa=0.9)
            assert abs(-(ep - em) / (2 * h) - F[r, d]) <= 1e-6 * np.abs(F[r]).max() + 1e-9


def test_full_rank_forces_equal_direct_forces():
    p = I.uniform(500, 241)
    q = I.rhs_uniform(500, 1, 242)[:, 0]
    o = O.Oracle(p, leaf_size=9, tol=0.0).compress()
    _, G = o.energy_forces(q)
    F = O.direct_forces_rows(p, q, np.arange(500))
    assert np.abs(-G - F).max() <= 1e-9 * np.abs(F).max()
