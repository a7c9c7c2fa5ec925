"""Skeleton storage (pivots + LU of K(sigma,tau), entries recomputed in FP64).

* FP64 handle: the product equals the oracle's skeleton-form product with the
  GPU's pivots to 1e-10 (cond K(sigma,tau) times rounding), and the factor-
  storage product of a handle built the same way to 1e-9.
* FP32 handle: within 1e-6 of the direct sum at tol 1e-7; several right-hand
  sides; forces work unchanged; the stored bytes are far below the factors'.
* The transpose product equals the oracle's skeleton transpose (FP64, 1e-10);
  the energy and its gradient follow from the two products.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def H(pts, **kw):
    import torch
    from paper_2307_16303_gb300.api import H3DMatrix
    return H3DMatrix(torch.from_numpy(np.ascontiguousarray(pts)).cuda(), **kw)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_skeleton_fp64_matches_oracle_and_factor_storage():
    import torch
    pts = I.uniform(8000, 271)
    kw = dict(leaf_size=32, tol=1e-6, precision="fp64")
    S = H(pts, storage="skeleton", **kw)
    F = H(pts, **kw)
    x = I.rhs_normal(8000, 1, 272)[:, 0]
    xt = torch.from_numpy(x).cuda()
    ys = S.matvec(xt).cpu().numpy()
    o = O.Oracle(pts, leaf_size=32, tol=1e-6).set_pivots(*S.export_pivots())
    assert rel(ys, o.matvec_skeleton(x)) <= 1e-10
    assert rel(ys, F.matvec(xt).cpu().numpy()) <= 1e-9
    assert S.stats()["factor_bytes"] < 0.5 * F.stats()["factor_bytes"]
    yT = S.matvec_T(xt).cpu().numpy()
    yTo = o.matvec_skeleton(x, transpose=True)
    assert rel(yT, yTo) <= 1e-10
    E, g = S.energy(xt)
    assert abs(E.item() - 0.5 * x @ ys) <= 1e-12 * abs(0.5 * x @ ys)
    assert rel(g.cpu().numpy(), 0.5 * (o.matvec_skeleton(x) + yTo)) <= 1e-10
    X3 = np.ascontiguousarray(np.stack([x, 2 * x, -x], axis=1))   # transpose in one 3-column pass
    YT3 = S.matvec_T(torch.from_numpy(X3).cuda()).cpu().numpy()
    assert rel(YT3[:, 1], 2 * yT) <= 1e-12


def test_skeleton_fp32_vs_direct_multi_rhs_and_forces():
    import torch
    n = 20000
    pts = I.uniform(n, 273)
    S = H(pts, leaf_size=64, tol=1e-7, precision="fp32", storage="skeleton")
    X = I.rhs_normal(n, 19, 274).astype(np.float32)   # a pass of 16 columns and one of 3
    Y = S.matvec(torch.from_numpy(X).cuda()).double().cpu().numpy()
    ref = O.direct(pts, X[:, [0, 15, 16, 18]].astype(np.float64))
    assert rel(Y[:, [0, 15, 16, 18]], ref) <= 1e-6
    y1 = S.matvec(torch.from_numpy(np.ascontiguousarray(X[:, 16])).cuda()).double().cpu().numpy()
    assert rel(Y[:, 16], y1) <= 1e-12   # the same FP64 sums in a pass of one column
    q = torch.from_numpy(I.rhs_uniform(n, 1, 275)[:, 0].astype(np.float32)).cuda()
    E, Fo = S.forces(q)
    rows = np.arange(0, n, 97)
    Fx = O.direct_forces_rows(pts, q.double().cpu().numpy(), rows)
    assert rel(Fo.cpu().numpy()[rows], Fx) <= 1e-5
