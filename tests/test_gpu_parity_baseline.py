"""Parity at the sizes of the benchmark workloads, through the C ABI.

* FP64, N = 65,536 uniform points, leaf 128, tol 1e-7 (depth 4): the product
  and the transpose product equal the oracle's Alg. 2 with the GPU's pivots
  frozen, to a relative 2-norm of 1e-12.  Its level-1 boxes hold ~8,192 points,
  so the source-side gather splits boxes into row tasks whose partial sums are
  reduced by a second kernel.
* N = 262,144 uniform points (seed 1), leaf 128, tol 1e-7, FP32 factors:
  the single-column product (CUDA cores) and the 32-column product (3xTF32 on
  the tensor cores) against the FP64 direct sum O1 on 4,096 seeded rows,
  column by column, to 1e-6; the transpose product of one column too.
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


@pytest.fixture(scope="module")
def fp64_65k():
    pts = I.uniform(65536, 1)
    A = H(pts, leaf_size=128, tol=1e-7, precision="fp64")
    o = O.Oracle(pts, leaf_size=128, tol=1e-7).set_pivots(*A.export_pivots())
    return pts, A, o


def test_fp64_65k_leaf128_depth_and_split_boxes(fp64_65k):
    pts, A, o = fp64_65k
    st = A.stats()
    assert st["depth"] == o.L == 4
    t = A.export_tree()
    lvl1 = t["box_end"][1:1 + t["nbox"][1]] - t["box_start"][1:1 + t["nbox"][1]]
    assert lvl1.max() > 4096      # taller than one row task of either gather path


def test_fp64_65k_forward_frozen_pivots(fp64_65k):
    pts, A, o = fp64_65k
    x = I.rhs_normal(65536, 1, 31)[:, 0]
    assert rel(gpu_apply(A, x), o.matvec(x)) <= 1e-12


def test_fp64_65k_transpose_frozen_pivots(fp64_65k):
    pts, A, o = fp64_65k
    x = I.rhs_uniform(65536, 1, 32)[:, 0]
    assert rel(gpu_apply(A, x, transpose=True), o.matvec(x, transpose=True)) <= 1e-12


@pytest.fixture(scope="module")
def cfg262k():
    pts = I.uniform(262144, 1)
    A = H(pts, leaf_size=128, tol=1e-7, precision="fp32_3xtf32")
    rows = I.sample_rows(262144, 4096, 4)
    return pts, A, rows


def test_262k_fp32_one_column_vs_direct(cfg262k):
    pts, A, rows = cfg262k
    x = I.rhs_normal(262144, 1, 2)[:, 0].astype(np.float32)
    y = gpu_apply(A, x)
    ref = O.direct_rows(pts, x.astype(np.float64), rows)
    assert rel(y[rows], ref) <= 1e-6
    yt = gpu_apply(A, x, transpose=True)
    assert rel(yt[rows], ref) <= 1e-6      # K is symmetric: A~^T x approximates the same sum


def test_262k_3xtf32_32_columns_vs_direct(cfg262k):
    pts, A, rows = cfg262k
    X = I.rhs_normal(262144, 32, 2).astype(np.float32)
    Y = gpu_apply(A, X)
    ref = O.direct_rows(pts, X.astype(np.float64), rows)
    for c in range(32):
        assert rel(Y[rows, c], ref[:, c]) <= 1e-6, c
