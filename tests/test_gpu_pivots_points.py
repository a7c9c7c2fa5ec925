"""Pivots imported into the GPU build, points moved with pivots frozen, and the
energy differentiated in the positions through autograd.

* h3d_import_pivots with the oracle's independently searched pivots (Alg. 1 on
  the CPU): the GPU then holds exactly those pivots, and its FP64 product and
  transpose product equal the oracle's Alg. 2 to 1e-12 -- frozen-pivot parity
  in the direction opposite to the other tests (there the oracle takes the
  GPU's pivots).  Skeleton storage: the same against the oracle's skeleton
  product (1e-10).  Invalid pivots are refused and leave the handle as it was.
* h3d_set_points: moving the points by a small displacement re-forms the
  factors at the new positions; the product equals the oracle built at the
  moved points with the same (frozen) pivots, whose tree is checked to be the
  same.  Unchanged coordinates change nothing; a non-finite one is refused.
* autograd: energy(A, q, points) gives dE/dq and dE/dp (= -F of h3d_forces)
  that match the oracle's cross-form gradient, and torch's gradcheck (central
  differences through h3d_set_points) passes in both inputs.
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


@pytest.mark.parametrize("N,leaf,tol,kern", [(20000, 40, 1e-7, "laplace"), (30000, 64, 1e-8, "laplace"),
                                             (6000, 32, 1e-8, "inv_r4")])
def test_import_oracle_pivots_fp64(N, leaf, tol, kern):
    pts = I.uniform(N, 301)
    A = H(pts, leaf_size=leaf, tol=tol, precision="fp64", kernel=kern)
    o = O.Oracle(pts, leaf_size=leaf, tol=tol, kernel=kern).compress()   # independent CPU search
    r, s, t = o.pivots()
    A.import_pivots(r, s, t)
    rg, sg, tg = A.export_pivots()
    assert np.array_equal(rg, r) and np.array_equal(sg, s) and np.array_equal(tg, t)
    x = I.rhs_normal(N, 1, 302)[:, 0]
    assert rel(gpu_apply(A, x), o.matvec(x)) <= 1e-12
    assert rel(gpu_apply(A, x, transpose=True), o.matvec(x, transpose=True)) <= 1e-12
    # several columns share a pass over the re-formed factors
    X = I.rhs_normal(N, 3, 303)
    Y = gpu_apply(A, X)
    Yo = o.matvec(X)
    for c in range(3):
        assert rel(Y[:, c], Yo[:, c]) <= 1e-12


def test_import_oracle_pivots_skeleton_and_fp32():
    pts = I.uniform(15000, 304)
    o = O.Oracle(pts, leaf_size=48, tol=1e-7).compress()
    piv = o.pivots()
    x = I.rhs_normal(15000, 1, 305)[:, 0]
    S = H(pts, leaf_size=48, tol=1e-7, precision="fp64", storage="skeleton")
    S.import_pivots(*piv)
    assert rel(gpu_apply(S, x), o.matvec_skeleton(x)) <= 1e-10
    assert rel(gpu_apply(S, x, transpose=True), o.matvec_skeleton(x, transpose=True)) <= 1e-10
    A32 = H(pts, leaf_size=48, tol=1e-7, precision="fp32")
    A32.import_pivots(*piv)
    assert rel(gpu_apply(A32, x.astype(np.float32)), o.matvec(x)) <= 1e-6


def test_import_rejects_invalid_pivots_and_keeps_handle():
    from paper_2307_16303_gb300.api import H3DError
    pts = I.uniform(8000, 306)
    A = H(pts, leaf_size=32, tol=1e-7, precision="fp64")
    x = I.rhs_normal(8000, 1, 307)[:, 0]
    y0 = gpu_apply(A, x)
    r, s, t = A.export_pivots()
    b = int(np.argmax(r >= 2))
    off = int(r[:b].sum())
    bad = [(r.copy(), s.copy(), t.copy()) for _ in range(3)]
    bad[0][1][off + 1] = bad[0][1][off]          # a row twice in one block
    bad[1][2][off] = -1                           # a column outside the block
    bad[2][0][b] = 10 ** 6                        # rank above min(m, n)
    for rr, ss, tt in bad[:2]:
        with pytest.raises(H3DError) as e:
            A.import_pivots(rr, ss, tt)
        assert e.value.status == 1
    with pytest.raises((H3DError, ValueError)):
        A.import_pivots(*bad[2])
    assert np.array_equal(gpu_apply(A, x), y0)
    # re-importing the handle's own pivots reproduces its product bit for bit
    A.import_pivots(r, s, t)
    assert np.array_equal(gpu_apply(A, x), y0)


@pytest.mark.parametrize("storage", ["factors", "skeleton"])
def test_set_points_reforms_at_moved_points(storage):
    import torch
    from paper_2307_16303_gb300.api import H3DError
    pts = I.uniform(12000, 308)
    A = H(pts, leaf_size=40, tol=1e-7, precision="fp64", storage=storage)
    piv = A.export_pivots()
    x = I.rhs_normal(12000, 1, 309)[:, 0]
    y0 = gpu_apply(A, x)
    A.set_points(torch.from_numpy(pts).cuda())          # the same coordinates: nothing changes
    assert np.array_equal(gpu_apply(A, x), y0)
    moved = pts + 1e-7 * np.random.default_rng(310).standard_normal(pts.shape)
    o = O.Oracle(moved, leaf_size=40, tol=1e-7)
    t0 = O.Oracle(pts, leaf_size=40, tol=1e-7).tree()
    assert np.array_equal(o.tree()["perm"], t0["perm"])    # no point crossed a box face
    o.set_pivots(*piv)
    A.set_points(torch.from_numpy(moved).cuda())
    y1 = gpu_apply(A, x)
    assert not np.array_equal(y1, y0)
    ref = o.matvec(x) if storage == "factors" else o.matvec_skeleton(x)
    assert rel(y1, ref) <= (1e-12 if storage == "factors" else 1e-10)
    bad = moved.copy()
    bad[5, 1] = np.nan
    with pytest.raises(H3DError) as e:
        A.set_points(torch.from_numpy(bad).cuda())
    assert e.value.status == 2
    assert np.array_equal(gpu_apply(A, x), y1)              # unchanged by the refused call


def test_autograd_energy_in_positions_and_charges():
    import torch
    from paper_2307_16303_gb300.autograd import energy
    n = 5000
    pts = I.uniform(n, 311)
    P = torch.from_numpy(pts).cuda().requires_grad_(True)
    from paper_2307_16303_gb300.api import H3DMatrix
    A = H3DMatrix(P, leaf_size=32, tol=1e-6, precision="fp64")
    qh = I.rhs_uniform(n, 1, 312)[:, 0]
    q = torch.from_numpy(qh).cuda().requires_grad_(True)
    E = energy(A, q, P)
    (2.0 * E).backward()
    o = O.Oracle(pts, leaf_size=32, tol=1e-6).set_pivots(*A.export_pivots())
    Eo, Go = o.energy_forces(qh)
    yo, yTo = o.matvec(qh), o.matvec(qh, transpose=True)
    assert abs(E.item() - 0.5 * qh @ yo) <= 1e-12 * abs(0.5 * qh @ yo)
    assert abs(E.item() - Eo) <= 1e-9 * abs(Eo)          # factor form vs cross form: rounding x cond
    assert rel(P.grad.cpu().numpy(), 2.0 * Go) <= 1e-8
    assert rel(q.grad.cpu().numpy(), yo + yTo) <= 1e-12
    # only what is asked for: charges without grad, positions with
    P.grad = None
    E2 = energy(A, q.detach(), P)
    E2.backward()
    assert rel(P.grad.cpu().numpy(), Go) <= 1e-8
    # against the exact forces of the dense energy on sampled points
    rows = I.sample_rows(n, 256, 313)
    Fx = O.direct_forces_rows(pts, qh, rows)
    assert rel(-P.grad.cpu().numpy()[rows], Fx) <= 1e-4


def test_autograd_gradcheck_positions_and_charges():
    import torch
    from paper_2307_16303_gb300.api import H3DMatrix
    from paper_2307_16303_gb300.autograd import energy
    n = 600
    pts = I.uniform(n, 314) * 0.9
    P = torch.from_numpy(pts).cuda().requires_grad_(True)
    A = H3DMatrix(P, leaf_size=16, tol=1e-6, precision="fp64")
    assert A.stats()["depth"] >= 2
    q = torch.from_numpy(I.rhs_uniform(n, 1, 315)[:, 0]).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda qq, pp: energy(A, qq, pp), (q, P), eps=1e-6, atol=1e-6, rtol=1e-4,
                                    fast_mode=True, nondet_tol=1e-9)   # forces add in FP64 atomics
    # the operator ends at the points it was built at
    A.set_points(P.detach())


def test_autograd_charges_only_without_requires_grad():
    import torch
    from paper_2307_16303_gb300.autograd import energy
    pts = I.uniform(3000, 316)
    A = H(pts, leaf_size=24, tol=1e-6, precision="fp64")
    q = torch.from_numpy(I.rhs_uniform(3000, 1, 317)[:, 0]).cuda()
    E = energy(A, q)                       # inference: q does not require grad
    assert not E.requires_grad
    assert E.item() == A.energy(q, grad=False).item()
