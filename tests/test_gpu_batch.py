"""Batched products of independent point clouds (h3d_batch_*).

Clouds of uneven size, half uniform in the cube and half on the unit sphere,
Laplace and Yukawa kernels alternating (the batched workload's recipe at small
sizes).  The graph replays the same kernels as separate products, so results
are compared bit for bit; new vectors re-capture; tuning keeps the results; two
clouds are checked against the direct sum.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SIZES = [3000, 9000, 5000, 12000, 4000, 7000]


def clouds():
    import torch
    from paper_2307_16303_gb300.api import H3DMatrix
    mats, pts = [], []
    for c, n in enumerate(SIZES):
        p = I.uniform(n, 300 + c) if c % 2 == 0 else I.sphere(n, 300 + c)
        kern = "laplace" if (c // 2) % 2 == 0 else "yukawa"
        pts.append((p, kern))
        mats.append(H3DMatrix(torch.from_numpy(p).cuda(), leaf_size=64, tol=1e-7, precision="fp32", kernel=kern))
    return mats, pts


def test_batch_matches_separate_products_bitwise():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch
    mats, pts = clouds()
    xs = [torch.from_numpy(I.rhs_normal(n, 1, 400 + c)[:, 0].astype(np.float32)).cuda() for c, n in enumerate(SIZES)]
    ys = [torch.empty_like(x) for x in xs]
    ref = [m.matvec(x) for m, x in zip(mats, xs)]
    B = H3DBatch(mats)
    for _ in range(2):                      # capture, then replay
        for y in ys:
            y.zero_()
        B.matvec(xs, ys)
        torch.cuda.synchronize()
        for y, r in zip(ys, ref):
            assert torch.equal(y, r)
    xs2 = [x * 0.5 + 1.0 for x in xs]        # new vectors: re-capture
    ys2 = [torch.empty_like(x) for x in xs2]
    B.matvec(xs2, ys2)
    torch.cuda.synchronize()
    for m, x, y in zip(mats, xs2, ys2):
        assert torch.equal(y, m.matvec(x))
    nb = B.tune(xs, ys)
    assert nb in (1, 2, 4)
    for y in ys:
        y.zero_()
    B.matvec(xs, ys)
    torch.cuda.synchronize()
    for y, r in zip(ys, ref):
        assert torch.equal(y, r)
    for c in (0, 3):                          # cube / Laplace and sphere / Yukawa
        p, kern = pts[c]
        d = O.direct(p, xs[c].double().cpu().numpy(), kernel=kern)
        assert np.linalg.norm(ys[c].double().cpu().numpy() - d) / np.linalg.norm(d) <= 1e-6
    B.free()
