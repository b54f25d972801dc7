"""``torch.autograd.Function`` around the propagator and its hand-written adjoint.

``evolve_potential(plan, V, psi0, dt, nsteps)`` returns ψ_n = U(Δt)^n ψ_0 for the lattice
plan with on-site potential V; its backward pass calls ``cheb_adjoint_potential`` (reverse
recurrence with √M checkpoints, see cheb_adjoint.cu) for dL/dV and dL/dψ_0.

PyTorch's gradient of a real loss with respect to a complex tensor z is 2 ∂L/∂z̄, while the
library's adjoint λ is ∂L/∂z̄; the conversion is a factor 2 each way.
"""
from __future__ import annotations

import torch

from ._cheb import Plan


class ChebEvolvePotential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, psi0, plan: Plan, dt: float, nsteps: int):
        plan.set_onsite(V.detach().contiguous())
        psi = psi0.detach().clone().contiguous()
        plan.evolve(psi, dt, nsteps)
        ctx.save_for_backward(V, psi0)
        ctx.plan = plan
        ctx.dt = dt
        ctx.nsteps = nsteps
        return psi

    @staticmethod
    def backward(ctx, grad_psi):
        V, psi0 = ctx.saved_tensors
        plan = ctx.plan
        plan.set_onsite(V.detach().contiguous())
        lam_n = (0.5 * grad_psi).contiguous()
        grad_V = torch.zeros_like(V, dtype=torch.float64)
        lam0 = torch.empty_like(psi0)
        plan.adjoint_potential(psi0.detach().contiguous(), ctx.dt, ctx.nsteps, lambda_n=lam_n,
                               grad=grad_V, lambda0=lam0)
        return grad_V.to(V.dtype), 2.0 * lam0, None, None, None


def evolve_potential(plan: Plan, V: torch.Tensor, psi0: torch.Tensor, dt: float, nsteps: int):
    return ChebEvolvePotential.apply(V, psi0, plan, dt, nsteps)
