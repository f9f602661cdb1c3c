"""Gradients of a freezing run through the hand-written adjoint of the FP64 step
(lbm_adjoint_fl_loss), exposed as a torch.autograd.Function.

The loss is L = sum_x (phi_pcm(x) f_l(x) - f_target(x))^2 after nsteps steps. Here
phi_pcm f_l is the liquid fraction of the phase-changing material, and phi_pcm is the
sum of phi_p over the phases with latent heat.  Its parameters theta = (T_wall, Ste, lam_ratio) are:
- the bottom wall temperature of the Dirichlet wall;
- the Stefan number, which sets L_p = c_p,s / Ste for every phase that changes
  phase (T_m - T_w,ref = 1);
- lambda_s / lambda_l of phase 0.

The library returns dL with respect to the coefficients, per side and per phase. This
module applies the chain rule to theta.  The adjoint runs when the forward is called:
the forward run is needed by it anyway, and backward only scales the stored gradient.
"""
from __future__ import annotations

import numpy as np

from . import lbm as L


def theta_gradient(case, g):
    """dL/d(T_wall, Ste, lam_ratio) from the coefficient gradient g (lbm_fl_grad) of a
    case built with those parameters.

    This is the chain rule of the caller's parameterisation of the loss, not a step of
    the method: the library differentiates with respect to the coefficients the step
    uses (wall temperatures, rho_l^p L_p, lambda_s^p, lambda_l^p); how a study maps its own
    parameters onto them (here L_p = c_p,s (T_m - T_w,ref) / Ste with T_m - T_w,ref = 1, and
    lambda_s^0 = lam_ratio lambda_l^0) is that study's choice, applied on the host."""
    ste = case.meta["ste"]
    d_ste = 0.0
    for p, ph in enumerate(case.phases):
        if ph["latent"] > 0.0:
            rhoL = ph["rho_l"] * ph["latent"]
            d_ste += g.rhoL[p] * (-rhoL / ste)          # rho_l L_p = rho_l c_p,s / Ste
    d_ratio = g.lambda_s[0] * case.phases[0]["lam_l"]   # lambda_s^0 = ratio lambda_l^0
    return np.array([g.T_wall[2], d_ste, d_ratio])


def run_adjoint(case, fl_target, nsteps, checkpoint_every=200, weight=None):
    """Loss and coefficient gradient of one FP64 run of `case` (fresh handle)."""
    s = L.Solver(case, precision="fp64")
    d = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    g = L.lbm_adjoint_fl_loss(s.h, d(case.phi), d(case.T), d(case.ux), d(case.uy), d(fl_target), d(weight),
                              L.LBM_HOST, nsteps, checkpoint_every)
    s.close()
    return g


def pcm_liquid_fraction(case, F):
    """phi_pcm f_l of exported fields F (phi_pcm = sum of phi_p over phases with L_p > 0)."""
    pcm = sum(F["phi"][p] for p, ph in enumerate(case.phases) if ph["latent"] > 0.0)
    return pcm * F["fl"]


def final_liquid_fraction(case, nsteps):
    """phi_pcm f_l after nsteps FP64 steps of `case` (e.g. the target run)."""
    s = L.Solver(case, precision="fp64").set_fields()
    s.step(nsteps)
    q = pcm_liquid_fraction(case, s.fields_numpy())
    s.close()
    return q


def _function():
    import torch

    class FreezeLoss(torch.autograd.Function):
        """loss = FreezeLoss.apply(theta, build, fl_target, nsteps, checkpoint_every)

        theta: tensor (T_wall, Ste, lam_ratio); build(T_wall=, ste=, lam_ratio=) -> Case."""

        @staticmethod
        def forward(ctx, theta, build, fl_target, nsteps, checkpoint_every):
            T_w, ste, ratio = [float(v) for v in theta.detach().cpu().double()]
            case = build(T_wall=T_w, ste=ste, lam_ratio=ratio)
            g = run_adjoint(case, fl_target, nsteps, checkpoint_every)
            ctx.save_for_backward(torch.tensor(theta_gradient(case, g), dtype=theta.dtype, device=theta.device))
            return torch.tensor(g.loss, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (gr,) = ctx.saved_tensors
            return grad_out * gr, None, None, None, None

    return FreezeLoss


_FreezeLoss = None


def FreezeLoss():
    """The torch.autograd.Function class (built on first use, so that importing this
    module does not import torch)."""
    global _FreezeLoss
    if _FreezeLoss is None:
        _FreezeLoss = _function()
    return _FreezeLoss
