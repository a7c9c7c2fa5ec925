"""Skeleton storage (pivots + LU of K(sigma,tau), entries recomputed in every product:
FP64 for FP64 handles, float-float on the FP32 pipes for FP32 handles of the
Laplace and 1/r^4 kernels).

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
    # a pass of one column takes the same entries and sums; the order of its
    # triangular solve differs, and its near field comes from the one-column
    # kernel instead of the eight-column one (FP32 sums in another order)
    assert rel(Y[:, 16], y1) <= 5e-7
    q = torch.from_numpy(I.rhs_uniform(n, 1, 275)[:, 0].astype(np.float32)).cuda()
    E, Fo = S.forces(q)
    rows = np.arange(0, n, 97)
    Fx = O.direct_forces_rows(pts, q.double().cpu().numpy(), rows)
    assert rel(Fo.cpu().numpy()[rows], Fx) <= 1e-5


@pytest.mark.parametrize("kern", ["laplace", "inv_r4", "yukawa"])
def test_skeleton_fp32_float_float_entries_vs_oracle(kern):
    # FP32 handles evaluate K(sigma,Y) and K(X,tau) of Laplace and 1/r^4 in
    # float-float on the FP32 pipes (Yukawa keeps FP64 entries); against the
    # oracle's FP64 skeleton product with the same pivots the difference is the
    # FP32 output and near field, not the entries
    import torch
    n = 12000
    pts = I.uniform(n, 276)
    kw = dict(leaf_size=48, tol=1e-7, kernel=kern)
    S = H(pts, precision="fp32", storage="skeleton", **kw)
    o = O.Oracle(pts, **kw).set_pivots(*S.export_pivots())
    x = I.rhs_normal(n, 1, 277)[:, 0].astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    x64 = x.astype(np.float64)
    assert rel(S.matvec(xt).double().cpu().numpy(), o.matvec_skeleton(x64)) <= 1e-6
    assert rel(S.matvec_T(xt).double().cpu().numpy(), o.matvec_skeleton(x64, transpose=True)) <= 1e-6
    X = np.ascontiguousarray(np.stack([x, -2 * x, 0.5 * x], axis=1))   # a 3-column pass
    Y = S.matvec(torch.from_numpy(X).cuda()).double().cpu().numpy()
    ref = o.matvec_skeleton(x64)
    for c, f in enumerate((1.0, -2.0, 0.5)):
        assert rel(Y[:, c], f * ref) <= 1e-6
    # moved points: the float-float coordinates follow
    moved = pts + 1e-7 * np.random.default_rng(278).standard_normal(pts.shape)
    om = O.Oracle(moved, **kw)
    assert np.array_equal(om.tree()["perm"], o.tree()["perm"])
    om.set_pivots(*S.export_pivots())
    S.set_points(torch.from_numpy(moved).cuda())
    assert rel(S.matvec(xt).double().cpu().numpy(), om.matvec_skeleton(x64)) <= 1e-6


def test_skeleton_fp32_float_float_close_pairs():
    # vertex-sharing leaf blocks hold point pairs much closer than the box size:
    # points clustered at box corners of the leaf level
    import torch
    rng = np.random.default_rng(279)
    corners = rng.integers(1, 8, size=(3000, 3)) * 0.25 - 1.0          # vertices of the level-3 grid
    pts = np.clip(corners + rng.uniform(-1e-3, 1e-3, size=corners.shape), -0.999, 0.999)
    kw = dict(leaf_size=16, tol=1e-7)
    S = H(pts, precision="fp32", storage="skeleton", **kw)
    S64 = H(pts, precision="fp64", storage="skeleton", **kw)
    x = I.rhs_normal(pts.shape[0], 1, 280)[:, 0].astype(np.float32)
    y32 = S.matvec(torch.from_numpy(x).cuda()).double().cpu().numpy()
    y64 = S64.matvec(torch.from_numpy(x.astype(np.float64)).cuda()).cpu().numpy()
    assert rel(y32, y64) <= 1e-6
