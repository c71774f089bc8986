"""torch.autograd wrapper of the transport map v -> m(1) (state equation, Sec. 2.1-2.2).

forward runs the library's semi-Lagrangian state solve (ga_transport). backward runs, by default, its
adjoint solve and body-force integral (ga_transport_vjp): the optimise-then-discretise gradient of
Sec. 2.1, not the exact derivative of the discrete forward map. With exact=True it runs the exact
vector-Jacobian product of the discrete map (ga_transport_vjp_exact; advection transport). Both run on
CUDA tensors of the problem's element type; there is no CPU path.
"""
from __future__ import annotations

import torch


class Transport(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, problem, exact=False):
        v = v.detach().contiguous()
        out = torch.empty(problem.shape, dtype=v.dtype, device=v.device)
        problem.transport(v, out)
        ctx.save_for_backward(v)
        ctx.problem = problem
        ctx.exact = exact
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (v,) = ctx.saved_tensors
        gv = torch.empty_like(v)
        ctx.problem.transport_vjp(v, grad_out.contiguous(), gv, exact=ctx.exact)
        return gv, None, None


def transport(v, problem, exact=False):
    """m(1) for velocity v (shape (dim, *n)); differentiable with respect to v (exact: the exact
    derivative of the discrete map instead of the optimise-then-discretise adjoint)."""
    return Transport.apply(v, problem, exact)
