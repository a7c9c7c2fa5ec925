"""Symmetric storage (each unordered admissible pair compressed once; the block
(Y,X) is the transpose of (X,Y), Eq. prank transposed), through the C ABI.

* FP64 frozen-pivot parity: with the GPU's pivots, the oracle's symmetric mode
  gives the same product to 1e-12, forward and transpose, at N = 20,000 leaf 32
  (many groups of small fused pairs per CTA, a ragged tail, pairs in the U / V
  layout) and at N = 65,536 leaf 128 (split source boxes); several columns
  (passes of 8) too.  The other direction: the oracle's independently searched
  symmetric pivots imported into the GPU build give the oracle's product to
  1e-12.
* FP32 at N = 262,144 (seed 1), leaf 128, tol 1e-7: one column and 19 columns
  against the FP64 direct sum O1 on 4,096 seeded rows to 1e-6, with fewer
  stored factor bytes than the ordered handle.
* The operator is symmetric: x^T A z = z^T A x, and the transpose product is the
  forward one.  Energy, its q-gradient and forces agree with the oracle's
  symmetric mode; moved points (pivots frozen) too.  Pivots that break the
  mirror relation are refused.  A batch holding a symmetric handle (graph form)
  gives the handle's own products.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def H(pts, **kw):
    import torch
    from paper_2307_16303_gb300.api import H3DMatrix
    return H3DMatrix(torch.from_numpy(np.ascontiguousarray(pts)).cuda(), **kw)


def gpu_apply(A, x, transpose=False):
    import torch
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda().to(A.dtype)
    y = A.matvec_T(xt) if transpose else A.matvec(xt)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


@pytest.mark.parametrize("N,leaf,tol,seed", [(20000, 32, 1e-6, 501), (65536, 128, 1e-7, 502)])
def test_symmetric_fp64_frozen_pivot_parity(N, leaf, tol, seed):
    pts = I.uniform(N, seed)
    A = H(pts, leaf_size=leaf, tol=tol, precision="fp64", storage="symmetric")
    P = H(pts, leaf_size=leaf, tol=tol, precision="fp64")
    o = O.Oracle(pts, leaf_size=leaf, tol=tol, symmetric=True).set_pivots(*A.export_pivots())
    x = I.rhs_normal(N, 1, seed + 1)[:, 0]
    y = gpu_apply(A, x)
    assert rel(y, o.matvec(x)) <= 1e-12
    assert rel(gpu_apply(A, x, transpose=True), o.matvec(x, transpose=True)) <= 1e-12
    # several columns: one pass of 8 and a ragged pass of 3
    X = I.rhs_normal(N, 11, seed + 2)
    Y = gpu_apply(A, X)
    Yo = o.matvec(X[:, [0, 7, 8, 10]])
    assert rel(Y[:, [0, 7, 8, 10]], Yo) <= 1e-12
    # the ordered handle's pivots are those of the primary blocks: close products,
    # and the symmetric handle stores markedly fewer factor bytes
    assert rel(y, gpu_apply(P, x)) <= 50 * tol
    sa, sp = A.stats(), P.stats()
    assert sa["factor_bytes"] < 0.8 * sp["factor_bytes"]
    assert sa["n_blocks"] == sp["n_blocks"] and sa["sum_rank"] > 0


def test_symmetric_imports_oracle_pivots():
    N, leaf, tol = 12000, 32, 1e-7
    pts = I.uniform(N, 503)
    o = O.Oracle(pts, leaf_size=leaf, tol=tol, symmetric=True).compress()   # independent CPU search
    A = H(pts, leaf_size=leaf, tol=tol, precision="fp64", storage="symmetric")
    A.import_pivots(*o.pivots())
    x = I.rhs_normal(N, 1, 504)[:, 0]
    assert rel(gpu_apply(A, x), o.matvec(x)) <= 1e-12
    # a mirror whose pivots are not its primary's swapped ones is refused, and
    # the handle keeps working
    r, s, t = o.pivots()
    lst = o.lists()
    b = int(np.nonzero((lst["tgt"] > lst["src"]) & (r >= 2))[0][0])
    off = int(np.sum(r[:b]))
    s2 = s.copy()
    s2[off], s2[off + 1] = s[off + 1], s[off]
    with pytest.raises(Exception):
        A.import_pivots(r, s2, t)
    assert rel(gpu_apply(A, x), o.matvec(x)) <= 1e-12


@pytest.fixture(scope="module")
def cfg2_sym():
    pts = I.uniform(262_144, 1)
    A = H(pts, leaf_size=128, tol=1e-7, storage="symmetric")
    rows = np.random.default_rng(505).choice(262_144, 4096, replace=False)
    return pts, A, rows


def test_symmetric_fp32_cfg2_vs_direct(cfg2_sym):
    pts, A, rows = cfg2_sym
    x = I.rhs_normal(262_144, 1, 506)[:, 0].astype(np.float32)
    y = gpu_apply(A, x)
    ref = O.direct_rows(pts, x.astype(np.float64), rows)
    assert rel(y[rows], ref) <= 1e-6
    X = I.rhs_normal(262_144, 19, 507).astype(np.float32)
    Y = gpu_apply(A, X)
    refX = O.direct_rows(pts, X[:, [0, 9, 18]].astype(np.float64), rows)
    for c, q in enumerate((0, 9, 18)):
        assert rel(Y[rows, q], refX[:, c]) <= 1e-6
    # at this size only the leaf level's pairs fit a stage (the level above has
    # ~512 points per box): fewer bytes, by less than at the 1M-point workload
    st = A.stats()
    P = H(pts, leaf_size=128, tol=1e-7)
    assert st["factor_bytes"] < 0.9 * P.stats()["factor_bytes"]
    P.free()


def test_symmetric_operator_is_symmetric(cfg2_sym):
    _, A, _ = cfg2_sym
    x = I.rhs_normal(262_144, 1, 508)[:, 0].astype(np.float32)
    z = I.rhs_normal(262_144, 1, 509)[:, 0].astype(np.float32)
    Ax, Az = gpu_apply(A, x), gpu_apply(A, z)
    a, b = float(z.astype(np.float64) @ Ax), float(x.astype(np.float64) @ Az)
    assert abs(a - b) <= 1e-6 * np.linalg.norm(Ax) * np.linalg.norm(z)
    assert rel(gpu_apply(A, x, transpose=True), Ax) <= 1e-6


def test_symmetric_energy_forces_and_moved_points():
    import torch
    N, leaf, tol = 8000, 32, 1e-8
    pts = I.uniform(N, 510)
    A = H(pts, leaf_size=leaf, tol=tol, precision="fp64", storage="symmetric")
    o = O.Oracle(pts, leaf_size=leaf, tol=tol, symmetric=True).set_pivots(*A.export_pivots())
    q = I.rhs_uniform(N, 1, 511)[:, 0]
    qt = torch.from_numpy(q).cuda()
    E, g = A.energy(qt)
    y = o.matvec(q)
    assert abs(E.item() - 0.5 * q @ y) <= 1e-12 * abs(0.5 * q @ y)
    assert rel(g.cpu().numpy(), y) <= 1e-12          # symmetric: the gradient is A~ q
    Ef, F = A.forces(qt)
    Eo, go = o.energy_forces(q)
    assert abs(Ef.item() - Eo) <= 1e-10 * abs(Eo)
    assert rel(-F.cpu().numpy(), go) <= 1e-8
    moved = pts + 1e-7 * np.random.default_rng(512).standard_normal(pts.shape)
    om = O.Oracle(moved, leaf_size=leaf, tol=tol, symmetric=True)
    assert np.array_equal(om.tree()["perm"], o.tree()["perm"])
    om.set_pivots(*A.export_pivots())
    A.set_points(torch.from_numpy(moved).cuda())
    assert rel(gpu_apply(A, q), om.matvec(q)) <= 1e-12


def test_symmetric_handle_in_a_batch():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch
    mats, xs = [], []
    for c, n in enumerate((9000, 15000, 4000)):
        p = I.uniform(n, 520 + c) if c != 1 else I.sphere(n, 520 + c)
        mats.append(H(p, leaf_size=48, tol=1e-7, storage="symmetric" if c != 2 else "factors"))
        xs.append(torch.from_numpy(I.rhs_normal(n, 1, 530 + c)[:, 0].astype(np.float32)).cuda())
    ys = [torch.empty_like(x) for x in xs]
    B = H3DBatch(mats)
    assert B.info()["persistent"] == -1      # the graph form only
    B.matvec(xs, ys)
    torch.cuda.synchronize()
    for m, x, y in zip(mats, xs, ys):
        r = m.matvec(x)
        assert rel(y.double().cpu().numpy(), r.double().cpu().numpy()) <= 1e-6
    B.free()
