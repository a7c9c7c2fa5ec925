"""GPU energy and gradient (h3d_energy, autograd) against the oracle and finite differences.

* FP64 handle, frozen pivots: E and dE/dq equal the oracle's to 1e-12.
* Central differences of the GPU energy match the GPU gradient (E is quadratic).
* autograd: backward of energy(A, q) gives the same gradient; torch's gradcheck
  (finite differences in FP64) passes on a small FP64 handle.
* FP32 handle at tol 1e-7: gradient within 1e-6 of the exact A q (direct sum).
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


def test_energy_fp64_frozen_matches_oracle():
    import torch
    pts = I.uniform(8000, 211)
    A = H(pts, leaf_size=32, tol=1e-6, precision="fp64")
    o = O.Oracle(pts, leaf_size=32, tol=1e-6).set_pivots(*A.export_pivots())
    q = I.rhs_uniform(8000, 1, 212)[:, 0]
    E, g = A.energy(torch.from_numpy(q).cuda())
    yo, yTo = o.matvec(q), o.matvec(q, transpose=True)
    Eo = 0.5 * q @ yo
    assert abs(E.item() - Eo) <= 1e-12 * abs(Eo)
    assert rel(g.cpu().numpy(), 0.5 * (yo + yTo)) <= 1e-12


def test_energy_central_differences_on_gpu():
    import torch
    pts = I.uniform(5000, 213)
    A = H(pts, leaf_size=24, tol=1e-5, precision="fp64")
    q = torch.from_numpy(I.rhs_uniform(5000, 1, 214)[:, 0]).cuda()
    _, g = A.energy(q)
    gmax = g.abs().max().item()
    for i in (0, 17, 999, 2500, 4999):
        h = 1e-3
        qp, qm = q.clone(), q.clone()
        qp[i] += h
        qm[i] -= h
        fd = (A.energy(qp, grad=False).item() - A.energy(qm, grad=False).item()) / (2 * h)
        assert abs(fd - g[i].item()) <= 1e-8 * gmax


def test_autograd_backward_and_gradcheck():
    import torch
    from paper_2307_16303_gb300.autograd import energy
    pts = I.uniform(3000, 215)
    A = H(pts, leaf_size=20, tol=1e-6, precision="fp64")
    q = torch.from_numpy(I.rhs_normal(3000, 1, 216)[:, 0]).cuda().requires_grad_(True)
    E = energy(A, q)
    (3.0 * E).backward()
    _, g = A.energy(q.detach())
    assert torch.equal(q.grad, 3.0 * g)
    small = H(I.uniform(300, 217), leaf_size=8, tol=1e-8, precision="fp64")
    qs = torch.from_numpy(I.rhs_normal(300, 1, 218)[:, 0]).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: energy(small, v), (qs,), eps=1e-4, atol=1e-7, rtol=1e-6)


def test_energy_fp32_gradient_vs_exact():
    import torch
    pts = I.uniform(20000, 219)
    A = H(pts, leaf_size=64, tol=1e-7, precision="fp32")
    q = I.rhs_uniform(20000, 1, 220)[:, 0].astype(np.float32)
    E, g = A.energy(torch.from_numpy(q).cuda())
    exact = O.direct(pts, q.astype(np.float64))
    assert rel(g.double().cpu().numpy(), exact) <= 1e-6
    Ee = 0.5 * q.astype(np.float64) @ exact
    assert abs(E.item() - Ee) <= 1e-6 * abs(Ee)
