"""GPU forces (h3d_forces) against the oracle and the exact dense forces.

* FP64 handles, pivots frozen (the oracle takes the GPU's): the energy equals
  the oracle's to 1e-10 and the forces its cross-form gradient to 1e-8.  Both
  are FP64 throughout; they differ in summation order and in the elimination of
  K(sigma, tau), whose condition (up to ~1e7 at tol 1e-6) scales the rounding of
  the solves: u * cond ~ 1e-9.
* FP32 handles evaluate only the near field in FP32 (entries to ~2e-7; the
  admissible blocks stay FP64): energy and forces within 1e-6 of the oracle's.
* Other kernels (Yukawa, 1/r^4, cos r / r): the same parity.
* The forces sum to zero (translation invariance with frozen pivots).
* Against the exact forces of the dense energy on sampled points (O1's
  gradient): within the compression error at tol 1e-7.
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


@pytest.mark.parametrize("prec,kern", [("fp64", "laplace"), ("fp32", "laplace"), ("fp64", "yukawa"),
                                       ("fp32", "yukawa"), ("fp64", "inv_r4"), ("fp64", "cos_r")])
def test_forces_match_oracle_frozen(prec, kern):
    import torch
    n = 6000
    pts = I.uniform(n, 251)
    kw = dict(leaf_size=32, tol=1e-6, kernel=kern)
    A = H(pts, precision=prec, **kw)
    q = I.rhs_uniform(n, 1, 252)[:, 0]
    qt = torch.from_numpy(q).cuda().to(A.dtype)
    E, F = A.forces(qt)
    o = O.Oracle(pts, **kw).set_pivots(*A.export_pivots())
    Eo, Go = o.energy_forces(qt.double().cpu().numpy())
    tE, tF = (1e-10, 1e-8) if prec == "fp64" else (1e-6, 1e-6)
    eF = rel(F.cpu().numpy(), -Go)
    print(f"{prec} {kern}: energy {abs(E.item() - Eo) / abs(Eo):.3e} forces {eF:.3e}")
    assert abs(E.item() - Eo) <= tE * abs(Eo)
    assert eF <= tF


def test_forces_sum_to_zero_and_match_exact():
    import torch
    n = 30000
    pts = I.uniform(n, 253)
    A = H(pts, leaf_size=64, tol=1e-7, precision="fp32")
    q = I.rhs_uniform(n, 1, 254)[:, 0].astype(np.float32)
    E, F = A.forces(torch.from_numpy(q).cuda())
    F = F.cpu().numpy()
    # zero up to rounding: this FP32 handle evaluates the two sides of each near
    # pair separately in FP32 (~1e-7 each)
    assert np.abs(F.sum(axis=0)).max() <= 1e-8 * np.abs(F).sum()
    rows = np.random.default_rng(255).choice(n, 512, replace=False)
    Fx = O.direct_forces_rows(pts, q.astype(np.float64), rows)
    err = rel(F[rows], Fx)
    assert err <= 1e-5, err
    # energies against the dense one, on the scale |q| |A q| / 2 of the quadratic
    # form (q ~ U(-1, 1) makes q^T A q itself much smaller by cancellation): the
    # cross form (FP64) and h3d_energy on this FP32 handle both to the
    # compression error of the product (~5e-7 relative at tol 1e-7)
    qd = q.astype(np.float64)
    y = O.direct(pts, qd)
    Ex, scale = 0.5 * qd @ y, 0.5 * np.linalg.norm(qd) * np.linalg.norm(y)
    assert abs(E.item() - Ex) <= 1e-6 * scale
    E2 = A.energy(torch.from_numpy(q).cuda(), grad=False).item()
    assert abs(E2 - Ex) <= 1e-6 * scale
