"""QAOA angle optimisation driven by the adjoint gradient.

§QAOA algorithm: the angles (gamma, beta) are tuned by a classical optimiser
so that the expected cut E(gamma, beta) = sum over edges of (1 - <Z_j Z_k>)/2
is as large as possible.  Here every start of a multi-start search is one
angle set of a gradient plan's batch, so one library call per iteration
evaluates E and dE/dgamma, dE/dbeta for all starts at once (the reverse
bucket sweep); the update itself is torch's Adam on the [B, p] angle tensors,
with a cosine-annealed step size so that the starts settle at stationary
points.
Nothing is evaluated on the CPU: the energy and its gradient come from the
plan's CUDA kernels through ``QAOAEnergy``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from .energy import EnergyPlan, qaoa_energy


@dataclass
class OptimizeResult:
    gamma: torch.Tensor            # [B, p] final angles of every start
    beta: torch.Tensor
    energy: torch.Tensor           # [B] expected cut at the final angles
    best: int                      # start with the largest final energy
    history: list = field(default_factory=list)  # [steps] list of the B energies (float64, CPU)


def maximize_cut(plan: EnergyPlan, gamma0: torch.Tensor, beta0: torch.Tensor, steps: int = 200,
                 lr: float = 0.02, record: bool = True) -> OptimizeResult:
    """Gradient ascent (Adam, step size annealed from lr to 0) on E for the B
    starts (gamma0, beta0) [B, p] of a
    gradient plan (``EnergyPlan(..., gradient=True)``).  Returns the final
    angles and energies and, if ``record``, the energy of every start at
    every iteration."""
    if not plan.options["gradient"]:
        raise ValueError("maximize_cut needs a plan created with gradient=True")
    gamma = gamma0.detach().clone().to(plan.device, torch.float64).requires_grad_(True)
    beta = beta0.detach().clone().to(plan.device, torch.float64).requires_grad_(True)
    opt = torch.optim.Adam([gamma, beta], lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=max(1, int(steps)))
    history = []
    for _ in range(int(steps)):
        opt.zero_grad(set_to_none=True)
        e = qaoa_energy(plan, gamma, beta)       # E[B] and, kept for backward, dE/dtheta[B, 2p]
        (-e.sum()).backward()                      # the starts are independent: one summed objective
        opt.step()
        sched.step()
        if record:
            history.append(e.detach().cpu())
    with torch.no_grad():
        e = plan.energy(gamma.detach(), beta.detach())
        plan.check()
    best = int(torch.argmax(e).item())
    return OptimizeResult(gamma=gamma.detach(), beta=beta.detach(), energy=e, best=best, history=history)
