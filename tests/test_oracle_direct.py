"""Pins for the oracle's kernel and direct sum (O1, Eq. Laplace3D).

Each value below is fixed by geometry or algebra, not by re-typing the oracle's
formula: closed-form potentials of symmetric point sets, the symmetry of K,
homogeneity of 1/r and 1/r^4 under scaling, and invariance under relabelling.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I

FOUR_PI = 4.0 * math.pi


def test_two_points_laplace_closed_form():
    d = 0.37
    p = np.array([[0.1, -0.2, 0.3], [0.1 + d, -0.2, 0.3]])
    x = np.array([2.0, -3.0])
    y = O.direct(p, x)
    np.testing.assert_allclose(y, [-3.0 / (FOUR_PI * d), 2.0 / (FOUR_PI * d)], rtol=1e-15)


def test_two_points_yukawa_closed_form():
    d, kappa = 0.5, 1.7
    p = np.array([[0.0, 0.0, 0.0], [0.0, 0.3, 0.4]])
    y = O.direct(p, np.array([1.0, 1.0]), kernel="yukawa", kappa=kappa)
    expect = math.exp(-kappa * d) / (FOUR_PI * d)
    np.testing.assert_allclose(y, [expect, expect], rtol=1e-15)


def test_cube_vertices_closed_form():
    # 8 vertices of a cube of side a: each sees 3 at a, 3 at a*sqrt2, 1 at a*sqrt3
    a = 0.6
    v = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float) * a - 0.3
    y = O.direct(v, np.ones(8))
    expect = (3 / a + 3 / (a * math.sqrt(2)) + 1 / (a * math.sqrt(3))) / FOUR_PI
    np.testing.assert_allclose(y, np.full(8, expect), rtol=1e-14)


def test_octahedron_closed_form_inv_r4():
    # 6 points at +-s e_k: 4 neighbours at s*sqrt2, one opposite at 2s
    s = 0.25
    p = np.concatenate([np.eye(3) * s, -np.eye(3) * s])
    y = O.direct(p, np.ones(6), kernel="inv_r4")
    expect = 4 / (s * math.sqrt(2)) ** 4 + 1 / (2 * s) ** 4
    np.testing.assert_allclose(y, np.full(6, expect), rtol=1e-14)


def test_cos_r_two_points():
    d = 0.9
    p = np.array([[0.0, 0.0, 0.0], [d, 0.0, 0.0]])
    y = O.direct(p, np.array([0.0, 1.0]), kernel="cos_r")
    np.testing.assert_allclose(y[0], math.cos(d) / d, rtol=1e-15)
    assert y[1] == 0.0


def test_zero_diagonal_and_coincident_points():
    p = np.array([[0.2, 0.2, 0.2], [0.2, 0.2, 0.2], [0.5, 0.2, 0.2]])
    y = O.direct(p, np.array([1.0, 10.0, 0.0]))
    # the coincident pair contributes nothing; the third point sees both at 0.3
    np.testing.assert_allclose(y[2], 11.0 / (FOUR_PI * 0.3), rtol=1e-14)
    assert y[0] == 0.0 and y[1] == 0.0


def test_symmetry_of_K():
    p = I.uniform(300, 11)
    x, z = I.rhs_normal(300, 2, 12).T
    lhs = z @ O.direct(p, x)
    rhs = x @ O.direct(p, z)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("kernel,power", [("laplace", 1), ("inv_r4", 4)])
def test_homogeneity_under_scaling(kernel, power):
    p = I.uniform(200, 3) * 0.4
    x = I.rhs_uniform(200, 1, 4)[:, 0]
    s = 0.5  # exact in binary, so scaled coordinates are exact
    y1 = O.direct(p, x, kernel=kernel)
    y2 = O.direct(p * s, x, kernel=kernel)
    np.testing.assert_allclose(y2, y1 / s ** power, rtol=1e-13)


def test_relabelling_invariance_and_rows_subset():
    p = I.uniform(257, 5)
    x = I.rhs_normal(257, 3, 6)
    perm = np.random.default_rng(7).permutation(257)
    y = O.direct(p, x)
    yp = O.direct(p[perm], x[perm])
    np.testing.assert_allclose(yp, y[perm], rtol=1e-13, atol=1e-13)
    rows = I.sample_rows(257, 40, 8)
    np.testing.assert_allclose(O.direct_rows(p, x, rows), y[rows], rtol=1e-15)
