"""torch.autograd.Function around the library's discrete adjoint.

``misfit(solver, u0, params, u_target, scheme="lawson_rk2", tau, nsteps, ckpt_every)``
returns J = 1/2 ||u(T) - u_target||^2 as a differentiable scalar tensor of
u0 (complex) and params = (nu, eta, gamma, kappa, zeta) (real, shape (5,)).
Forward and backward both run in libfcgle.so (fcgle_adjoint computes the loss
and the gradients in one call); gradients follow PyTorch's convention for a
real loss of a complex input, dJ/dRe u0 + i dJ/dIm u0.
"""
import torch

from . import fcgle


class _Misfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, params, u_target, solver, scheme, tau, nsteps, ckpt_every):
        p = [float(x) for x in params.detach().cpu().tolist()]
        solver.set_coefficients(*p)
        loss, g, gp = solver.adjoint(scheme, tau, nsteps, u0.detach(), u_target.detach(), ckpt_every)
        ctx.save_for_backward(g, torch.tensor(gp, dtype=params.dtype, device=params.device))
        return torch.tensor(loss, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gJ):
        g, gp = ctx.saved_tensors
        return (gJ.to(g.real.dtype) * g, gJ.to(gp.dtype) * gp, None, None, None, None, None, None)


def misfit(solver, u0, params, u_target, scheme="lawson_rk2", tau=1e-3, nsteps=1, ckpt_every=25):
    return _Misfit.apply(u0, params, u_target, solver, scheme, tau, nsteps, ckpt_every)
