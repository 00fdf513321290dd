"""torch.autograd.Function around the butterfly: forward bf_apply, backward bf_apply_adjoint.

For the complex linear map f = B g, PyTorch's gradient convention (conjugate
Wirtinger) makes the vector-Jacobian product grad_g = B^H grad_f, which is the
exact adjoint butterfly (every step of the forward conjugate-transposed, levels in
reverse).  Both directions run in the sm_103a kernels.
"""
from __future__ import annotations

import torch


class ButterflyApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, plan):
        ctx.plan = plan
        return plan.apply(g.contiguous())

    @staticmethod
    def backward(ctx, grad_f):
        return ctx.plan.apply_adjoint(grad_f.contiguous()), None


def butterfly(g: torch.Tensor, plan) -> torch.Tensor:
    """Differentiable f = B g (g: CUDA tensor of shape (N^d,) or (nrhs, N^d))."""
    return ButterflyApply.apply(g, plan)


def cgls(plan, d: torch.Tensor, iters: int = 20):
    """CGLS on the normal equations B^H B m = B^H d (Hestenes-Stiefel form, m0 = 0).

    Returns m and the residual norms ||B m_k - d|| for k = 0..iters (non-increasing in
    exact arithmetic).  Each iteration applies B once and B^H once.
    """
    m = torch.zeros_like(d)
    r = d.clone()                              # r = d - B m
    s = plan.apply_adjoint(r)                  # s = B^H r
    p = s.clone()
    gamma = torch.vdot(s.flatten(), s.flatten()).real
    hist = [torch.linalg.vector_norm(r).item()]
    for _ in range(iters):
        q = plan.apply(p)
        qq = torch.vdot(q.flatten(), q.flatten()).real
        if qq == 0:
            break
        alpha = gamma / qq
        m = m + alpha * p
        r = r - alpha * q
        s = plan.apply_adjoint(r)
        gamma_new = torch.vdot(s.flatten(), s.flatten()).real
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        hist.append(torch.linalg.vector_norm(r).item())
    return m, hist
