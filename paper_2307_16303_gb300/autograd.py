"""Differentiation of the HODLR3D energy through the C ABI.

``energy(A, q, points=None)`` returns E = 1/2 q^T A~ q as a differentiable 0-d
tensor of the charges q and, when ``points`` is given, of the point positions:

* forward: ``h3d_energy`` without the gradient (one product A~ q and the FP64
  reduction).  With ``points``, the operator is first moved to those
  coordinates (``h3d_set_points``: tree, lists and ACA pivots frozen, factors
  re-formed; a no-op when they are the coordinates it already holds).
* backward, only for the inputs that need it:
  dE/dq = 1/2 (A~ + A~^T) q   (``h3d_energy`` with the gradient: the product
  and the transpose product), and
  dE/dp = -F                   (``h3d_forces``: the near-field gradient plus
  the cross form K(X,tau) K(sigma,tau)^{-1} K(sigma,Y) of every admissible
  block differentiated with the pivots frozen, Sec. 4.1 Eq. prank).
Every product, reduction and gradient runs in the library's kernels; this
module only passes tensors.
"""
import torch


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, points, A):
        if points is not None:
            A.set_points(points)
        E = A.energy(q, grad=False)
        ctx.A = A
        ctx.save_for_backward(q, points if points is not None else q.new_empty(0))
        ctx.has_points = points is not None
        return E

    @staticmethod
    def backward(ctx, gE):
        q, points = ctx.saved_tensors
        A = ctx.A
        if ctx.has_points:
            A.set_points(points)      # the coordinates of this forward (no-op if unchanged)
        gq = gp = None
        if ctx.needs_input_grad[0]:
            _, g = A.energy(q, grad=True)
            gq = gE.to(g.dtype) * g
        if ctx.has_points and ctx.needs_input_grad[1]:
            _, F = A.forces(q)
            gp = -gE.to(F.dtype) * F
        return gq, gp, None


def energy(A, q, points=None):
    """E = 1/2 q^T A~ q for the H3DMatrix ``A`` and charges ``q`` (N,),
    differentiable in q and, if ``points`` ((N, 3) float64 CUDA tensor) is given,
    in the positions, with the operator's tree and ACA pivots frozen."""
    return _Energy.apply(q, points, A)
