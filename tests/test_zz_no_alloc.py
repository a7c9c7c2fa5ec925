"""The no-allocation Morton-order entry point gives the same keys and order as
the regular build.

h3d_morton_order_noalloc exists for callers that cannot allocate device memory
(a host application that owns a fixed memory pool, a plugin handed only
pre-allocated buffers): its scratch is a fixed static array inside the library.
This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.  It must pass alone in a fresh
process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2307_16303_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2307_16303_gb300 import api, build_ext
    build_ext.build()
    return api


def _noalloc(api, pts_dev, n, lo=(-1.0, -1.0, -1.0), side=2.0):
    import torch
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    lo_a = (ctypes.c_double * 3)(*lo)
    st = api.lib().h3d_morton_order_noalloc(pts_dev.data_ptr(), n, lo_a, side, keys.data_ptr(), perm.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    return st, keys.cpu().numpy().view(np.uint64), perm.cpu().numpy().astype(np.int64)


def _oracle_order(pts, lo=(-1.0, -1.0, -1.0), side=2.0):
    """The oracle's Morton keys and the stable order by (key, original index)."""
    from oracle import oracle as O
    keys = O.morton(pts, lo=lo, side=side)
    perm = np.argsort(keys, kind="stable")
    return keys[perm], perm


def test_noalloc_order_matches_oracle_twice_in_a_row():
    import torch
    api = _lib()
    # two clouds, one call each, back to back, against the oracle's keys and a
    # stable sort of them; a second call must not see the first call's scratch
    for pts in (I.uniform(300_000, 84), I.jittered_grid(40, 85)):
        st, keys, perm = _noalloc(api, torch.from_numpy(pts).cuda(), pts.shape[0])
        assert st == 0
        ok, op = _oracle_order(pts)
        assert np.array_equal(keys, ok)
        assert np.array_equal(perm, op)


def test_noalloc_order_matches_build_twice_in_a_row():
    import torch
    api = _lib()
    # two different clouds, one call each, back to back: the second call must not
    # see anything left in the shared scratch by the first
    for pts, leaf in ((I.uniform(300_000, 81), 64), (I.sphere(50_000, 82) * 0.999, 32)):
        dev = torch.from_numpy(pts).cuda()
        st, keys, perm = _noalloc(api, dev, pts.shape[0])
        assert st == 0
        A = api.H3DMatrix(dev, leaf_size=leaf, tol=1e-5, precision="fp32")
        ref = A.export_tree()
        A.free()
        assert np.array_equal(keys, ref["keys"])
        assert np.array_equal(perm, ref["perm"])


def test_noalloc_rejects_bad_sizes_and_points():
    import torch
    api = _lib()
    maxn = 1 << 20
    dev = torch.zeros((maxn + 1, 3), dtype=torch.float64, device="cuda")
    st, _, _ = _noalloc(api, dev, maxn + 1)
    assert st == 1                       # beyond the fixed scratch: H3D_ERR_ARG
    st, _, _ = _noalloc(api, dev, 0)
    assert st == 1
    bad = torch.from_numpy(np.array([[0.0, 0.0, 0.0], [0.0, 2.5, 0.0]])).cuda()
    st, _, _ = _noalloc(api, bad, 2)
    assert st == 2                       # H3D_ERR_DOMAIN
    # host buffers are refused before any launch (H3D_ERR_ARG)
    host_pts = np.ascontiguousarray(I.uniform(100, 86))
    keys = torch.empty(100, dtype=torch.int64, device="cuda")
    perm = torch.empty(100, dtype=torch.int32, device="cuda")
    lo_a = (ctypes.c_double * 3)(-1.0, -1.0, -1.0)
    s = torch.cuda.current_stream().cuda_stream
    st = api.lib().h3d_morton_order_noalloc(host_pts.ctypes.data, 100, lo_a, 2.0, keys.data_ptr(), perm.data_ptr(), s)
    assert st == 1
    hkeys = np.zeros(100, np.uint64)
    dpts = torch.from_numpy(host_pts).cuda()
    st = api.lib().h3d_morton_order_noalloc(dpts.data_ptr(), 100, lo_a, 2.0, hkeys.ctypes.data, perm.data_ptr(), s)
    assert st == 1
    # the largest accepted size works and agrees with the oracle's keys and a
    # stable sort of them
    pts = I.uniform(maxn, 83)
    st, keys, perm = _noalloc(api, torch.from_numpy(pts).cuda(), maxn)
    assert st == 0
    ok, op = _oracle_order(pts)
    assert np.array_equal(keys, ok)
    assert np.array_equal(perm, op)
