"""Batched products of independent point clouds (h3d_batch_*).

Clouds of uneven size, half uniform in the cube and half on the unit sphere,
Laplace and Yukawa kernels alternating (the batched workload's recipe at small
sizes), plus degenerate members (one leaf, no far field).

* Graph form: it replays the same kernels as separate products, so results are
  compared bit for bit; new vectors re-capture.
* Persistent form: every item is computed by one CTA in a fixed order, so the
  result is the same bits on every run and for every CTA count; it differs from
  the separate products only in summation order (FP32: a few units of 1e-7;
  FP64: 1e-13); two clouds are checked against the direct sum (Alg. 2 against
  the dense product at tol 1e-7).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SIZES = [3000, 9000, 5000, 12000, 4000, 7000]


def clouds(precision="fp32", sizes=SIZES, leaf=64):
    import torch
    from paper_2307_16303_gb300.api import H3DMatrix
    mats, pts = [], []
    for c, n in enumerate(sizes):
        p = I.uniform(n, 300 + c) if c % 2 == 0 else I.sphere(n, 300 + c)
        kern = "laplace" if (c // 2) % 2 == 0 else "yukawa"
        pts.append((p, kern))
        mats.append(H3DMatrix(torch.from_numpy(p).cuda(), leaf_size=leaf, tol=1e-7, precision=precision, kernel=kern))
    return mats, pts


def vectors(sizes, dtype, seed=400):
    import torch
    return [torch.from_numpy(I.rhs_normal(n, 1, seed + c)[:, 0].astype(dtype)).cuda() for c, n in enumerate(sizes)]


def rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run(B, xs, ys):
    import torch
    for y in ys:
        y.fill_(float("nan"))
    B.matvec(xs, ys)
    torch.cuda.synchronize()
    return [y.clone() for y in ys]


def test_graph_form_matches_separate_products_bitwise():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch
    mats, pts = clouds()
    xs = vectors(SIZES, np.float32)
    ys = [torch.empty_like(x) for x in xs]
    ref = [m.matvec(x) for m, x in zip(mats, xs)]
    B = H3DBatch(mats)
    B.set_mode(False)
    assert B.info()["persistent"] == 0
    for _ in range(2):                      # capture, then replay
        for y, r in zip(run(B, xs, ys), ref):
            assert torch.equal(y, r)
    xs2 = [x * 0.5 + 1.0 for x in xs]        # new vectors: re-capture
    ys2 = [torch.empty_like(x) for x in xs2]
    for m, x, y in zip(mats, xs2, run(B, xs2, ys2)):
        assert torch.equal(y, m.matvec(x))
    for c in (0, 3):                          # cube / Laplace and sphere / Yukawa
        p, kern = pts[c]
        d = O.direct(p, xs[c].double().cpu().numpy(), kernel=kern)
        assert np.linalg.norm(ref[c].double().cpu().numpy() - d) / np.linalg.norm(d) <= 1e-6
    B.free()


def test_persistent_form_fp32():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch, H3DError
    mats, pts = clouds()
    xs = vectors(SIZES, np.float32)
    ys = [torch.empty_like(x) for x in xs]
    ref = [m.matvec(x) for m, x in zip(mats, xs)]
    B = H3DBatch(mats)
    info = B.info()
    assert info["persistent"] == 1 and info["ctas_per_sm"] >= 2   # the default form
    first = run(B, xs, ys)
    for _ in range(3):                        # same bits every run
        for y, f in zip(run(B, xs, ys), first):
            assert torch.equal(y, f)
    for y, r in zip(first, ref):
        assert rel(y, r) <= 2e-6
    for c in (0, 3):
        p, kern = pts[c]
        d = O.direct(p, xs[c].double().cpu().numpy(), kernel=kern)
        assert np.linalg.norm(first[c].double().cpu().numpy() - d) / np.linalg.norm(d) <= 1e-6
    xs2 = [x * 0.5 + 1.0 for x in xs]        # new vectors: pointers copied to the device
    ys2 = [torch.empty_like(x) for x in xs2]
    for m, x, y in zip(mats, xs2, run(B, xs2, ys2)):
        assert rel(y, m.matvec(x)) <= 2e-6
    nb = B.tune(xs, ys)
    assert nb in (0, 1, 2, 4)
    B.set_mode(True)                          # any item size and CTA count: the same bits
    for y, f in zip(run(B, xs, ys), first):
        assert torch.equal(y, f)
    with pytest.raises(H3DError):             # a handle twice would share its scratch
        H3DBatch([mats[0], mats[1], mats[0]])
    B.free()


def test_persistent_form_same_bits_for_every_cta_count():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch
    mats, _ = clouds(sizes=SIZES[:4])
    xs = vectors(SIZES[:4], np.float32)
    ys = [torch.empty_like(x) for x in xs]
    B = H3DBatch(mats)
    B.set_mode(True, 1)
    assert B.info()["ctas_per_sm"] == 1
    first = run(B, xs, ys)
    # a CTA count, item size or queue order changes only which CTA runs an item
    # and when, never how it is computed
    for cps, ng, lg, lag in ((2, 0, 0, -1), (3, 8, 1, 0), (64, 4, 4, 1), (5, 1, 3, 8), (7, 4, 2, 2)):
        B.set_mode(True, cps, ng, lg, lag)
        for y, f in zip(run(B, xs, ys), first):
            assert torch.equal(y, f)
    assert 2 <= B.info()["ctas_per_sm"] < 64          # capped at the occupancy limit
    B.free()


def test_persistent_form_fp64_and_degenerate_members():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch
    sizes = [6000, 40, 2500, 9000]             # 40 points: one leaf, no far field
    mats, pts = clouds("fp64", sizes)
    xs = vectors(sizes, np.float64, 500)
    ys = [torch.empty_like(x) for x in xs]
    ref = [m.matvec(x) for m, x in zip(mats, xs)]
    B = H3DBatch(mats)
    assert B.info()["persistent"] == 1
    for y, r in zip(run(B, xs, ys), ref):
        assert rel(y, r) <= 1e-13
    p, kern = pts[1]
    d = O.direct(p, xs[1].cpu().numpy(), kernel=kern)
    assert np.linalg.norm(ys[1].cpu().numpy() - d) / np.linalg.norm(d) <= 1e-14
    B.free()


def test_mixed_precision_batch_uses_the_graph_form():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch, H3DError, H3DMatrix
    p0, p1 = I.uniform(3000, 310), I.sphere(2000, 311)
    mats = [H3DMatrix(torch.from_numpy(p0).cuda(), leaf_size=64, tol=1e-7, precision="fp32"),
            H3DMatrix(torch.from_numpy(p1).cuda(), leaf_size=64, tol=1e-7, precision="fp64")]
    xs = [torch.from_numpy(I.rhs_normal(3000, 1, 1)[:, 0].astype(np.float32)).cuda(),
          torch.from_numpy(I.rhs_normal(2000, 1, 2)[:, 0]).cuda()]
    ys = [torch.empty_like(x) for x in xs]
    B = H3DBatch(mats)
    assert B.info()["persistent"] == -1
    with pytest.raises(H3DError):
        B.set_mode(True)
    for m, x, y in zip(mats, xs, run(B, xs, ys)):
        assert torch.equal(y, m.matvec(x))
    B.free()


def test_tuner_item_shapes_per_size_and_rank_bucket():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch
    sizes = [4000, 40000, 6000, 150000]        # three size buckets
    mats, pts = clouds(sizes=sizes, leaf=64)
    xs = vectors(sizes, np.float32, 600)
    ys = [torch.empty_like(x) for x in xs]
    B = H3DBatch(mats)
    B.set_mode(True)
    first = run(B, xs, ys)
    ng0, lg0 = B.groups()
    assert set(ng0) == {4} and set(lg0) == {2}      # the default shape for every operator
    B.tune(xs, ys)
    ng, lg = B.groups()
    shapes = {(2, 1), (4, 1), (4, 2), (8, 2), (8, 4), (16, 4)}
    assert all((int(a), int(b)) in shapes for a, b in zip(ng, lg))
    # operators of one bucket share a shape (clouds 0 and 2 are both below 2^15 points)
    if mats[0].stats()["max_rank"] <= 96 and mats[2].stats()["max_rank"] <= 96:
        assert (ng[0], lg[0]) == (ng[2], lg[2])
    B.set_mode(True)                                  # the tuned shapes: the same bits
    for y, f in zip(run(B, xs, ys), first):
        assert torch.equal(y, f)
    q = B.queue()
    for o in range(len(sizes)):                       # the queue follows each operator's shape
        near = q[(q[:, 0] == o) & (q[:, 1] == 1)]
        leaf = q[(q[:, 0] == o) & (q[:, 1] == 3)]
        assert near[:, 3].max() == min(int(ng[o]), mats[o].stats()["n_leaves"])
        assert leaf[:, 3].max() == min(int(lg[o]), mats[o].stats()["n_leaves"])
        assert near[:, 3].sum() == mats[o].stats()["n_leaves"] == leaf[:, 3].sum()
    B.free()
