"""F_p as a torch.autograd.Function over the CUDA kernels.

    F = p_objective(U, graph, p)          # Eq. 1, a 0-d float64 tensor
    F.backward()                          # U.grad = dF/dU   (gradient kernel)
    torch.autograd.grad(..., create_graph=True) then differentiate again:
                                          # Hessian-vector products (HVP kernel)

The gradient of F is computed by pspec_eval; the derivative of the gradient
applied to a cotangent V is the exact Hessian applied to V (pspec_hvp), which
is its own transpose because the Hessian is symmetric and block diagonal over
columns.  Nothing here stores per-edge state: every backward re-runs the edge
kernels on U.
"""
from __future__ import annotations

import torch


class _Gradient(torch.autograd.Function):
    """U -> grad F(U); its backward is V -> H(U) V."""

    @staticmethod
    def forward(ctx, U, graph, p):
        _, grad = graph.eval(U, p)
        ctx.save_for_backward(U)
        ctx.graph, ctx.p = graph, p
        return grad

    @staticmethod
    def backward(ctx, gG):
        (U,) = ctx.saved_tensors
        HV = ctx.graph.hvp(U, gG.contiguous().to(U.dtype), ctx.p)
        return HV, None, None


class FpFunction(torch.autograd.Function):
    """U -> F_p(U) (Eq. 1).  Backward: the gradient kernel; double backward:
    the Hessian-vector-product kernel."""

    @staticmethod
    def forward(ctx, U, graph, p):
        F, grad = graph.eval(U, p)
        ctx.save_for_backward(U, grad)
        ctx.graph, ctx.p = graph, p
        return F.reshape(())

    @staticmethod
    def backward(ctx, gF):
        U, grad = ctx.saved_tensors
        if torch.is_grad_enabled():  # create_graph: keep the gradient differentiable
            grad = _Gradient.apply(U, ctx.graph, ctx.p)
        return gF.to(grad.dtype) * grad, None, None


def p_objective(U, graph, p):
    """F_p(U) with autograd support (first and second order)."""
    return FpFunction.apply(U, graph, float(p))
