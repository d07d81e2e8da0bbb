"""torch.autograd.Function around the library's hand-written adjoint (ade_adjoint).

``misfit(sim, C0, theta, target, nsteps, ckpt_every)`` returns J = 1/2 |C^N - C*|^2 after nsteps
predictor-corrector steps (Eq. 8-9) started from C0 with dispersivities theta = (alpha_L, alpha_T,
D_m) and a fixed time step; ``J.backward()`` delivers dJ/dC0 (on the GPU, float32) and dJ/dtheta
(float64).  Forward and gradient both run in libade_sph.so; this module only moves tensors.
"""
from __future__ import annotations

import torch


class DispersivityMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, C0, theta, sim, target, nsteps, ckpt_every):
        sim.C.copy_(C0.detach().to(sim.C.device, torch.float32))
        th = theta.detach().to("cpu", torch.float64).tolist()
        sim.set_dispersivity(th[0], th[1], th[2])
        J, g, dC0, _ = sim.adjoint(target, nsteps, ckpt_every, want_dC0=True)
        ctx.save_for_backward(dC0.clone(), torch.tensor(g, dtype=torch.float64))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dC0, g = ctx.saved_tensors
        gJ = gJ.detach()
        return (gJ.to(dC0.device, torch.float32) * dC0, gJ.cpu() * g, None, None, None, None)


def misfit(sim, C0, theta, target, nsteps, ckpt_every=40):
    return DispersivityMisfit.apply(C0, theta, sim, target, nsteps, ckpt_every)
