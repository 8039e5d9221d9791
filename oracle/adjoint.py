"""Discrete adjoint of the collide-and-stream scheme by reverse-mode automatic
differentiation of the oracle's own FP64 forward (test infrastructure).

The paper runs no adjoint; this is the plain definition of the gradient of the
final-time density misfit J = 1/2 sum_x (rho(x, T) - rho*(x))^2 with respect to the
initial fields (populations start at f^eq of those fields) and the shared relaxation
time tau_LB of the conserved fields.  All intermediate states are kept (small grids).
"""
from __future__ import annotations

import torch

F64 = torch.float64


def misfit_and_grad(make_scheme, Q_init, target, n_steps, tau_cons):
    """make_scheme(tau_cons_tensor) -> Scheme.  Returns (J, dJ/dQ_init, dJ/dtau)."""
    Qi = Q_init.clone().to(F64).requires_grad_(True)
    tc = torch.tensor(float(tau_cons), dtype=F64, requires_grad=True)
    sch = make_scheme(tc)
    f = sch.init(Qi)
    for n in range(n_steps):
        f = sch.step(f, n * sch.dt)
    rho = sch.moments(f)[0]
    J = 0.5 * ((rho - target) ** 2).sum()
    gQ, gt = torch.autograd.grad(J, [Qi, tc])
    return float(J), gQ.detach(), float(gt)


def misfit(make_scheme, Q_init, target, n_steps, tau_cons):
    with torch.no_grad():
        sch = make_scheme(torch.tensor(float(tau_cons), dtype=F64))
        f = sch.init(Q_init.to(F64))
        for n in range(n_steps):
            f = sch.step(f, n * sch.dt)
        rho = sch.moments(f)[0]
        return float(0.5 * ((rho - target) ** 2).sum())
