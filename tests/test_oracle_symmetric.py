"""Pins for the oracle's symmetric storage (each unordered admissible pair
compressed once; the mirror block (Y,X) takes the transposed factors and the
swapped pivots, which is Eq. prank transposed for a symmetric kernel).

* The operator it applies is an exactly symmetric matrix (bit for bit), while
  the ordered mode's is symmetric only to the ACA tolerance.
* Its primary blocks carry exactly the ordered mode's pivots (the same ACA on
  the same block), and every mirror the swapped pivots of its primary.
* Its product is as close to the dense sum O1 as the ordered mode's, its
  transpose product equals its forward product, and its energy gradient
  matches the ordered mode's to the tolerance.
* Frozen pivots that break the mirror relation are refused.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dense(o, n):
    return o.matvec(np.eye(n))


@pytest.mark.parametrize("kern", ["laplace", "yukawa"])
def test_symmetric_operator_is_exactly_symmetric(kern):
    pts = I.uniform(900, 401)
    kw = dict(kernel=kern, leaf_size=12, tol=1e-5)
    S = O.Oracle(pts, symmetric=True, **kw).compress()
    P = O.Oracle(pts, **kw).compress()
    assert S.L >= 3
    A = dense(S, 900)
    B = dense(P, 900)
    assert np.array_equal(A, A.T)
    # the ordered mode compresses (X,Y) and (Y,X) separately: not exactly symmetric
    asym = np.abs(B - B.T).max() / np.abs(B).max()
    assert 0.0 < asym < 1e-3


def test_primary_pivots_equal_ordered_and_mirrors_swapped():
    pts = I.uniform(3000, 402)
    S = O.Oracle(pts, leaf_size=24, tol=1e-7, symmetric=True).compress()
    P = O.Oracle(pts, leaf_size=24, tol=1e-7).compress()
    lst = S.lists()
    rs, ss, ts = S.pivots()
    rp, sp, tp = P.pivots()
    offs = np.concatenate([[0], np.cumsum(rs)])
    offp = np.concatenate([[0], np.cumsum(rp)])
    key = {(l, t, s): b for b, (l, t, s) in enumerate(zip(lst["level"], lst["tgt"], lst["src"]))}
    nprim = 0
    for b, (l, t, s) in enumerate(zip(lst["level"], lst["tgt"], lst["src"])):
        if t < s:
            nprim += 1
            assert rs[b] == rp[b]
            assert np.array_equal(ss[offs[b]:offs[b + 1]], sp[offp[b]:offp[b + 1]])
            assert np.array_equal(ts[offs[b]:offs[b + 1]], tp[offp[b]:offp[b + 1]])
        else:
            p = key[(l, s, t)]
            assert rs[b] == rs[p]
            assert np.array_equal(ss[offs[b]:offs[b + 1]], ts[offs[p]:offs[p + 1]])
            assert np.array_equal(ts[offs[b]:offs[b + 1]], ss[offs[p]:offs[p + 1]])
    assert 2 * nprim == S.n_blocks


def test_mirror_factors_are_transposed_primaries():
    pts = I.uniform(2000, 403)
    S = O.Oracle(pts, leaf_size=20, tol=1e-6, symmetric=True).compress()
    lst = S.lists()
    key = {(l, t, s): b for b, (l, t, s) in enumerate(zip(lst["level"], lst["tgt"], lst["src"]))}
    checked = 0
    for b in range(0, S.n_blocks, 37):
        l, t, s = lst["level"][b], lst["tgt"][b], lst["src"][b]
        p = key[(l, s, t)]
        Ub, Vb = S.block_factors(b)
        Up, Vp = S.block_factors(p)
        assert np.array_equal(Ub, Vp) and np.array_equal(Vb, Up)
        # and the block is the kernel block to the tolerance
        xs, m, ys, n = S.block_geometry(b)
        sp = S.sorted_points()
        d = np.linalg.norm(sp[xs:xs + m, None, :] - sp[None, ys:ys + n, :], axis=2)
        K = 1.0 / (4.0 * np.pi * d)   # admissible boxes are disjoint: d > 0
        assert np.linalg.norm(Ub @ Vb.T - K) <= 1e-4 * np.linalg.norm(K)
        checked += 1
    assert checked > 10


@pytest.mark.parametrize("kern", ["laplace", "inv_r4"])
def test_symmetric_product_error_vs_direct(kern):
    pts = I.uniform(6000, 404)
    x = I.rhs_normal(6000, 1, 405)[:, 0]
    y = O.direct(pts, x, kernel=kern)
    for tol in (1e-5, 1e-7):
        es = rel(O.Oracle(pts, kernel=kern, leaf_size=48, tol=tol, symmetric=True).compress().matvec(x), y)
        eo = rel(O.Oracle(pts, kernel=kern, leaf_size=48, tol=tol).compress().matvec(x), y)
        assert es < 10 * tol
        assert eo / 3 < es < 3 * eo


def test_symmetric_transpose_equals_forward_and_energy_gradient():
    pts = I.uniform(2500, 406)
    S = O.Oracle(pts, leaf_size=24, tol=1e-8, symmetric=True).compress()
    P = O.Oracle(pts, leaf_size=24, tol=1e-8).compress()
    x = I.rhs_normal(2500, 1, 407)[:, 0]
    assert rel(S.matvec(x, transpose=True), S.matvec(x)) <= 1e-14
    q = I.rhs_uniform(2500, 1, 408)[:, 0]
    Es, gs = S.energy_forces(q)
    Ep, gp = P.energy_forces(q)
    assert abs(Es - Ep) <= 1e-7 * abs(Ep)
    assert rel(gs, gp) <= 1e-6


def test_frozen_pivots_must_respect_the_mirror():
    pts = I.uniform(1500, 409)
    S = O.Oracle(pts, leaf_size=16, tol=1e-6, symmetric=True).compress()
    r, s, t = S.pivots()
    # the same pivots frozen again are accepted and give the same product
    x = I.rhs_normal(1500, 1, 410)[:, 0]
    F = O.Oracle(pts, leaf_size=16, tol=1e-6, symmetric=True).set_pivots(r, s, t)
    assert np.array_equal(F.matvec(x), S.matvec(x))
    # a mirror whose pivots differ from its primary's swapped ones is refused
    lst = S.lists()
    b = int(np.nonzero((lst["tgt"] > lst["src"]) & (r >= 2))[0][0])
    off = int(np.sum(r[:b]))
    s2 = s.copy()
    s2[off], s2[off + 1] = s[off + 1], s[off]
    with pytest.raises(O.OracleError):
        O.Oracle(pts, leaf_size=16, tol=1e-6, symmetric=True).set_pivots(r, s2, t)
    # and the switch is refused once pivots exist
    with pytest.raises(O.OracleError):
        O._check(O._load().h3do_set_symmetric(S._h, 0))
