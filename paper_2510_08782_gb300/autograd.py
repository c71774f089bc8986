"""torch.autograd wrapper of the transport map v -> m(1) (state equation, Sec. 2.1-2.2).

forward runs the library's semi-Lagrangian state solve (ga_transport); backward runs its adjoint
solve and body-force integral (ga_transport_vjp), i.e. the optimise-then-discretise gradient of
Sec. 2.1, not the exact derivative of the discrete forward map. Both run on CUDA tensors of the
problem's element type; there is no CPU path.
"""
from __future__ import annotations

import torch


class Transport(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, problem):
        v = v.detach().contiguous()
        out = torch.empty(problem.shape, dtype=v.dtype, device=v.device)
        problem.transport(v, out)
        ctx.save_for_backward(v)
        ctx.problem = problem
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (v,) = ctx.saved_tensors
        gv = torch.empty_like(v)
        ctx.problem.transport_vjp(v, grad_out.contiguous(), gv)
        return gv, None


def transport(v, problem):
    """m(1) for velocity v (shape (dim, *n)); differentiable with respect to v."""
    return Transport.apply(v, problem)
