"""PyTorch differentiation of the registration objective J(u) of Eq. (11).

``objective(ctx, u)`` returns J as a 0-d float64 CUDA tensor that
participates in autograd: its backward is the library's hand-written adjoint
(``ngf_gradient``: P^T [dT/dy (G^T (2 r a))] for the NGF term of Eq. (1) plus
the curvature, volume-change and keypoint adjoints), evaluated at the saved u.
The forward pass runs the objective-only kernel; the backward pass recomputes
the warped template and its derivative on the fly, so nothing per voxel is
kept between the two (``eager=True`` evaluates J and the gradient in one fused
pass instead and keeps only the grid-sized gradient).

``gn_hvp(ctx, u, v)`` is the Gauss-Newton Hessian-vector product
H(u) v = (H_D + alpha H_R + gamma H_V + delta H_K) v, the matrix the solver
uses (not the exact Hessian, and without a second backward pass).

Shapes: u, v are float32 CUDA tensors (3, mz, my, mx) in mm, as for
``api.Context``.
"""
from __future__ import annotations

import torch

__all__ = ["objective", "objective_terms", "gn_hvp"]


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(fctx, u, ctx, eager):
        u = u.detach().contiguous()
        if eager:
            terms, grad = ctx.ngf_gradient(u)
            fctx.save_for_backward(grad)
        else:
            terms = ctx.ngf_objective(u)
            fctx.save_for_backward(u)
        fctx.ctx, fctx.eager = ctx, eager
        return terms[4].clone()

    @staticmethod
    def backward(fctx, gJ):
        (saved,) = fctx.saved_tensors
        grad = saved if fctx.eager else fctx.ctx.ngf_gradient(saved)[1]
        return (gJ.to(grad.dtype) * grad, None, None)


def objective(ctx, u, eager=False):
    """J(u) (Eq. 11) as a differentiable 0-d float64 tensor; +inf on a fold."""
    return _Objective.apply(u, ctx, eager)


def objective_terms(ctx, u):
    """(D, R, V, K, J) as a float64 tensor (no autograd)."""
    return ctx.ngf_objective(u.detach().contiguous())


def gn_hvp(ctx, u, v, relinearize=True):
    """H(u) v with the Gauss-Newton matrix at u (re-linearises at u unless told not to)."""
    if relinearize:
        ctx.gn_linearize(u.detach().contiguous(), want_grad=False)
    return ctx.gn_matvec(v.detach().contiguous())
