"""torch.autograd.Function around the C ABI: y = A(k) sigma with a hand-written backward.

Forward calls ``ifgf_apply_ws`` on a workspace tensor it keeps: afterwards that
tensor holds the forward state (w sigma in Morton order and every level's cone
values).  Backward calls ``ifgf_apply_vjp_ws`` on it, which returns A^H grad_y
(the gradient with respect to the density) and Re <grad_y, dA/dk sigma> (the
gradient with respect to the wavenumber k, with the plan's octree and cone
structure frozen and eta held fixed) without a second forward apply.
complex128 densities use the FP64 path, complex64 the mixed path.
"""
from __future__ import annotations

import torch

from .binding import Plan


class IFGFApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma: torch.Tensor, k: torch.Tensor, plan: Plan):
        if abs(float(k) - plan.params.k) > 1e-12 * max(1.0, abs(plan.params.k)):
            raise ValueError("k must equal the plan's wavenumber (build a plan per k)")
        ctx.plan = plan
        y, state = plan.apply_with_state(sigma)
        ctx.save_for_backward(k, state)
        ctx.squeeze = sigma.dim() == 1
        return y

    @staticmethod
    def backward(ctx, grad_y: torch.Tensor):
        k, state = ctx.saved_tensors
        gs, dk = ctx.plan.vjp_from_state(state, grad_y.contiguous(), with_dk=ctx.needs_input_grad[1])
        gk = torch.tensor(dk, dtype=k.dtype, device=k.device) if ctx.needs_input_grad[1] else None
        return gs if ctx.needs_input_grad[0] else None, gk, None


def ifgf_apply(sigma: torch.Tensor, k: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable y = A(k) sigma (see IFGFApply)."""
    return IFGFApply.apply(sigma, k, plan)
