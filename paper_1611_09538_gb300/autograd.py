"""torch.autograd front end of the SE1P evaluation (argument marshalling only).

  se1p_energy(plan, x, q)    -> U = 1/2 sum q phi; backward: dU/dx = -F, dU/dq = phi
                                 (both computed by the forward evaluation)
  se1p_potential(plan, x, q) -> phi; backward through se1p_eval_vjp (adjoint evaluation
                                 with the cotangent as charges, grid recomputed)

x is [n,3] float64 and q is [n] float64 on the plan's CUDA device.  The
derivatives are those of the discrete SE1P approximation, which is what the
kernels evaluate; for a neutral system dq is meaningful only for neutral
charge changes (the q-gradient is defined up to a constant shift).
"""
from __future__ import annotations

import torch

from . import se1p


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, plan):
        r = plan.eval(x.detach().contiguous(), q.detach().contiguous())
        ctx.save_for_backward(r.phi, r.force)
        return r.energy[0]

    @staticmethod
    def backward(ctx, gU):
        phi, F = ctx.saved_tensors
        return -gU * F, gU * phi, None


class _Potential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, plan):
        xd, qd = x.detach().contiguous(), q.detach().contiguous()
        r = plan.eval(xd, qd)
        ctx.save_for_backward(xd, qd)
        ctx.plan = plan
        return r.phi

    @staticmethod
    def backward(ctx, v):
        x, q = ctx.saved_tensors
        n = x.shape[0]
        gx = torch.empty_like(x)
        gq = torch.empty_like(q)
        se1p.se1p_eval_vjp(ctx.plan.handle, n, x, q, v.contiguous(), gx, gq)
        code = se1p.se1p_plan_sync_status(ctx.plan.handle)
        if code != 0:
            raise se1p.SE1PError(code, "se1p_eval_vjp (device status)")
        return gx, gq, None


def se1p_energy(plan: se1p.Plan, x: torch.Tensor, q: torch.Tensor) -> torch.Tensor:
    """Differentiable energy U = 1/2 sum q phi (scalar tensor)."""
    return _Energy.apply(x, q, plan)


def se1p_potential(plan: se1p.Plan, x: torch.Tensor, q: torch.Tensor) -> torch.Tensor:
    """Differentiable potentials phi [n]."""
    return _Potential.apply(x, q, plan)
