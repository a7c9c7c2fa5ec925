"""Failure detection without a GPU fault.

* A bounded device wait that runs out: the persistent batch kernel is given a
  queue from which one gather item of the first operator is left out, so that
  operator's reduce and leaf items wait on a completion counter that nothing
  will complete.  With the wait limit set to 1 ms, the launch stops, the next
  call reports H3D_ERR_TIMEOUT once, and the batch and the handles then give the
  same results as before.
* Allocation failure: with the library's allocation-failure hook, every
  device allocation of a build in turn is made to fail; each build returns
  H3D_ERR_OOM and releases everything it allocated (the free device memory
  returns to its level before the call).  A failure inside the first energy
  call's scratch allocation leaves the handle usable.
"""
import numpy as np
import pytest

from paper_2307_16303_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_batch_wait_runs_out_then_recovers():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch, H3DError, H3DMatrix
    sizes = (20000, 12000)
    mats = [H3DMatrix(torch.from_numpy(I.uniform(n, 400 + k)).cuda(), leaf_size=64, tol=1e-6, precision="fp32")
            for k, n in enumerate(sizes)]
    xs = [torch.from_numpy(I.rhs_normal(n, 1, 410 + k)[:, 0].astype(np.float32)).cuda() for k, n in enumerate(sizes)]
    ys = [torch.empty_like(x) for x in xs]
    B = H3DBatch(mats)
    assert B.info()["persistent"] == 1
    B.set_mode(True)
    B.matvec(xs, ys)
    torch.cuda.synchronize()
    ref = [y.clone() for y in ys]
    q = B.queue()
    g0 = int(np.flatnonzero((q[:, 0] == 0) & (q[:, 1] == 0))[0])     # a gather item of operator 0
    B.set_wait_limit(1_000_000)                                      # 1 ms
    B.set_queue(np.delete(q, g0, axis=0))
    B.matvec(xs, ys)                      # returns at once; the kernel's wait runs out
    torch.cuda.synchronize()
    with pytest.raises(H3DError) as e:
        B.matvec(xs, ys)                  # the next call reports it ...
    assert e.value.status == 6
    B.set_queue(None)                     # ... once; the complete queue works again
    B.set_wait_limit(2_000_000_000)
    B.matvec(xs, ys)
    torch.cuda.synchronize()
    for y, r in zip(ys, ref):
        assert torch.equal(y, r)
    y0 = mats[0].matvec(xs[0])
    torch.cuda.synchronize()
    assert torch.allclose(y0, ref[0], rtol=0, atol=2e-6 * ref[0].abs().max().item())
    B.free()


def test_batch_queue_items_are_checked():
    import torch
    from paper_2307_16303_gb300.api import H3DBatch, H3DError, H3DMatrix
    A = H3DMatrix(torch.from_numpy(I.uniform(5000, 420)).cuda(), leaf_size=64, tol=1e-6, precision="fp32")
    B = H3DBatch([A])
    q = B.queue()
    for bad in ([1, 0, 0, 1], [0, 0, 10 ** 6, 1], [0, 3, 0, 10 ** 6], [0, 7, 0, 1], [0, 4, -1, 0]):
        with pytest.raises(H3DError) as e:
            B.set_queue(np.array([bad], np.int32))
        assert e.value.status == 1
    assert np.array_equal(B.queue(), q)
    for ns in (0, 999, 10 ** 12):
        with pytest.raises(H3DError):
            B.set_wait_limit(ns)
    B.free()


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failure_releases_everything():
    import torch
    from paper_2307_16303_gb300 import api
    pts = torch.from_numpy(I.uniform(4000, 430)).cuda()
    api.H3DMatrix(pts, leaf_size=32, tol=1e-6, precision="fp64").free()   # warm-up
    base = _free_bytes()
    failures = 0
    try:
        for k in range(400):
            api.debug_fail_alloc(k)
            try:
                A = api.H3DMatrix(pts, leaf_size=32, tol=1e-6, precision="fp64")
            except api.H3DError as e:
                assert e.status == 3, (k, e.status)
                failures += 1
                assert _free_bytes() == base, k
                continue
            A.free()
            del A
            break
        else:
            pytest.fail("the build never completed")
    finally:
        api.debug_fail_alloc(-1)
    assert failures >= 20                 # every allocation of the build was made to fail once
    assert _free_bytes() == base
    # a failure in a product's first-use scratch: the handle stays usable
    A = api.H3DMatrix(pts, leaf_size=32, tol=1e-6, precision="fp64")
    q = torch.from_numpy(I.rhs_uniform(4000, 1, 431)[:, 0]).cuda()
    for k in range(3):
        api.debug_fail_alloc(k)
        with pytest.raises(api.H3DError) as e:
            A.energy(q)
        assert e.value.status == 3
    api.debug_fail_alloc(-1)
    E, g = A.energy(q)
    y, yT = A.matvec(q), A.matvec_T(q)
    assert torch.allclose(g, 0.5 * (y + yT), rtol=0, atol=1e-12 * g.abs().max().item())
