"""Pins for the oracle's ACA (Sec. 4.1, Eqs. prank / LR).

* With tolerance 0 the cross approximation reaches full rank and reproduces the
  block (exact up to rounding).
* The approximant interpolates the pivot rows and columns exactly.
* U V^T equals the skeleton form K(X,tau) K(sigma,tau)^{-1} K(sigma,Y) of
  Eq. prank, evaluated independently with a dense solve.
* The approximation error is of the order of the tolerance, and Eckart-Young
  bounds it from below by the (r+1)-st singular value.
* Ranks by interaction class follow Table "rankgrowth" / Theorem 1 in shape:
  well-separated ranks stay nearly flat as boxes grow, vertex ranks exceed them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I


def dense_block(pts, xs, m, ys, n):
    """The kernel block built in numpy from the sorted points (zero when r = 0)."""
    a = pts[xs:xs + m][:, None, :]
    b = pts[ys:ys + n][None, :, :]
    r = np.sqrt(((a - b) ** 2).sum(-1))
    with np.errstate(divide="ignore"):
        k = 1.0 / (4.0 * math.pi * r)
    k[r == 0] = 0.0
    return k


@pytest.fixture(scope="module")
def small():
    o = O.Oracle(I.uniform(1500, 51), leaf_size=24, tol=1e-8)
    o.compress()
    return o


def test_full_rank_reproduces_block():
    o = O.Oracle(I.uniform(600, 52), leaf_size=40, tol=0.0)
    o.compress()
    sp = o.sorted_points()
    rank, _, _ = o.pivots()
    for b in range(0, o.n_blocks, max(1, o.n_blocks // 25)):
        xs, m, ys, n = o.block_geometry(b)
        U, V = o.block_factors(b)
        K = dense_block(sp, xs, m, ys, n)
        assert rank[b] == min(m, n)
        assert np.linalg.norm(K - U @ V.T) <= 1e-12 * np.linalg.norm(K)


def test_interpolates_pivots_and_matches_skeleton_form(small):
    o = small
    sp = o.sorted_points()
    rank, sig, tau = o.pivots()
    off = np.concatenate([[0], np.cumsum(rank)])
    for b in range(0, o.n_blocks, max(1, o.n_blocks // 40)):
        xs, m, ys, n = o.block_geometry(b)
        r = int(rank[b])
        s, t = sig[off[b]:off[b] + r], tau[off[b]:off[b] + r]
        assert len(set(s)) == r and len(set(t)) == r
        U, V = o.block_factors(b)
        K = dense_block(sp, xs, m, ys, n)
        A = U @ V.T
        scale = np.abs(K).max()
        # the residual vanishes on pivot rows and columns
        assert np.abs((K - A)[s, :]).max() <= 1e-12 * scale
        assert np.abs((K - A)[:, t]).max() <= 1e-12 * scale
        # Eq. prank: K(X,tau) K(sigma,tau)^{-1} K(sigma,Y)
        skel = K[:, t] @ np.linalg.solve(K[np.ix_(s, t)], K[s, :])
        assert np.linalg.norm(A - skel) <= 1e-9 * np.linalg.norm(K)


def test_error_of_order_tol_and_eckart_young(small):
    o = small
    sp = o.sorted_points()
    rank, _, _ = o.pivots()
    worst = 0.0
    for b in range(0, o.n_blocks, max(1, o.n_blocks // 60)):
        xs, m, ys, n = o.block_geometry(b)
        U, V = o.block_factors(b)
        K = dense_block(sp, xs, m, ys, n)
        E = K - U @ V.T
        rel = np.linalg.norm(E) / np.linalg.norm(K)
        worst = max(worst, rel)
        sv = np.linalg.svd(K, compute_uv=False)
        r = int(rank[b])
        if r < min(m, n):
            assert sv[r] <= np.linalg.norm(E, 2) * (1 + 1e-9)
    assert worst <= 50 * o.tol


def test_frozen_own_pivots_give_identical_product(small):
    o = small
    x = I.rhs_normal(o.N, 2, 53)
    y1 = o.matvec(x)
    r, s, t = o.pivots()
    o2 = O.Oracle(o.points, leaf_size=24, tol=1e-8).set_pivots(r, s, t)
    assert np.array_equal(o2.matvec(x), y1)


def test_rank_cap_is_reported():
    o = O.Oracle(I.uniform(1500, 54), leaf_size=24, tol=1e-14, rank_cap=3)
    with pytest.raises(O.OracleError) as e:
        o.compress()
    assert e.value.status == 5


def test_rank_growth_by_class():
    # Table "rankgrowth": K(I_X, I_W) ranks do not grow with N, K(I_X, I_V) grow
    # slowly; vertex ranks exceed well-separated ones at the same box size.
    o = O.Oracle(I.uniform(32768, 1), leaf_size=64, tol=1e-7).compress()
    rank, _, _ = o.pivots()
    li = o.lists()

    def mean(level, cls):
        sel = (li["level"] == level) & (li["cls"] == cls)
        return rank[sel].mean()

    w2, w3 = mean(2, 4), mean(3, 4)   # 512 vs 64 points per box
    v2, v3 = mean(2, 3), mean(3, 3)
    assert w2 / w3 < 1.5              # 8x more points, nearly the same rank
    assert v2 > w2 and v3 > w3
    assert v2 / v3 < 2.0              # slower than the N^(1/3) of edge interactions
    assert rank[li["level"] == 1].max() < 0.05 * 4096
