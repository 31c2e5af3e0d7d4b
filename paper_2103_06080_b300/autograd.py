"""torch.autograd.Function around kzk_advance / kzk_adjoint.

Forward advances a copy of u0 by n_steps ExpRK22 steps and keeps the spectral
state every `ckpt_every` steps inside the plan; backward returns the gradient
with respect to u0 through the library's hand-written adjoint (transposed
WENO5 including the derivatives of the nonlinear weights, conjugated
phi-multipliers, adjoint FFTs), recomputing each segment from its checkpoint.
The plan holds one set of checkpoints: run backward before the next forward
through the same plan.  This is what a shape-optimisation loop
over the initial pressure profile needs: d loss(u(sigma_end)) / d u0.
"""
from __future__ import annotations

import torch


class KZKAdvance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, plan, n_steps: int, sigma0: float = 0.0, ckpt_every: int = 32):
        u = u0.detach().clone().contiguous()
        plan.advance_checkpointed(u, n_steps, sigma0, ckpt_every)
        ctx.plan = plan
        return u

    @staticmethod
    def backward(ctx, g):
        g0 = ctx.plan.adjoint_checkpointed(g.contiguous())
        return g0, None, None, None, None


def advance(u0: torch.Tensor, plan, n_steps: int, sigma0: float = 0.0, ckpt_every: int = 32) -> torch.Tensor:
    """Differentiable propagation u(sigma0 + n_steps dsigma) from u0."""
    return KZKAdvance.apply(u0, plan, n_steps, sigma0, ckpt_every)
