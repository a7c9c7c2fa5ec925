"""Differentiation of the HODLR3D energy through the C ABI.

``energy(A, q)`` returns E = 1/2 q^T A~ q as a differentiable 0-d tensor: the
forward pass runs ``h3d_energy`` (the product A~ q, the transpose product A~^T q,
the FP64 reduction and the gradient 1/2 (A~ + A~^T) q, all in the library's
kernels); the backward pass hands the stored gradient to autograd, scaled by
the incoming gradient.  A~ itself (the points and the compressed factors) is
not a differentiable input here.
"""
import torch


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, A):
        E, g = A.energy(q, grad=q.requires_grad)
        ctx.save_for_backward(g if g is not None else q.new_empty(0))
        return E

    @staticmethod
    def backward(ctx, gE):
        (g,) = ctx.saved_tensors
        return gE.to(g.dtype) * g, None


def energy(A, q):
    """E = 1/2 q^T A~ q for the H3DMatrix ``A`` and charges ``q`` (N,), differentiable in q."""
    return _Energy.apply(q, A)
