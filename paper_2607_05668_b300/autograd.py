"""torch.autograd.Function around the library's hand-written adjoint (lbx_adjoint).

DensityMisfit.apply(Q_init, tau, rho_target, make_scheme, n_steps, ckpt_every) returns
J = 1/2 sum_x (rho(x, T) - rho*(x))^2 as a 0-d float64 tensor.  Its backward gives
dJ/dQ_init and dJ/dtau (tau = tau_LB of the conserved fields).  The forward call runs the
forward sweep and the GPU reverse sweep together (the reverse sweep recomputes segments
from the forward's checkpoints), so backward only scales the stored gradients.
"""
import torch

from . import lbx


class DensityMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q_init, tau, rho_target, make_scheme, n_steps, ckpt_every):
        sch = make_scheme(float(tau))
        J, gQ, gt = lbx.adjoint(sch, Q_init.detach().cpu(), n_steps, ckpt_every, rho_target.detach().cpu())
        ctx.save_for_backward(gQ.to(Q_init.device), torch.tensor(gt, dtype=torch.float64, device=tau.device))
        return torch.tensor(J, dtype=torch.float64, device=Q_init.device)

    @staticmethod
    def backward(ctx, gJ):
        gQ, gt = ctx.saved_tensors
        return gJ * gQ, gJ * gt, None, None, None, None
