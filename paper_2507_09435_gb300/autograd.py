"""torch.autograd wrapper of one implicit load step and its adjoint.

``ImplicitStep.apply(gs, step, E_p, phi_p)`` solves the load step ``step`` of
the GPU scene ``gs`` from its committed state with per-particle Young's
modulus ``E_p`` and friction angle ``phi_p`` (1-D float64 tensors in the
caller's particle order) and returns the particle displacement increments
``du_p`` (np x dim).  The step stays staged (not committed): ``backward``
calls ``mpm_adjoint`` on it with dL/d(du_p), and the caller commits with
``gs.commit()`` when it is done.  Only argument marshalling happens here;
the solve and the adjoint run in libmpm's kernels.
"""
from __future__ import annotations

import numpy as np
import torch


class ImplicitStep(torch.autograd.Function):

    @staticmethod
    def forward(ctx, gs, step, E_p, phi_p):
        gs.set_params(E_p=E_p.detach().cpu().double().numpy(), phi_p=phi_p.detach().cpu().double().numpy())
        gs.solve_staged(step)
        du = gs.particle_increment()[:, :gs.dim]
        ctx.gs = gs
        ctx.dev = E_p.device
        return torch.from_numpy(np.ascontiguousarray(du)).to(E_p.device)

    @staticmethod
    def backward(ctx, grad_du):
        gs = ctx.gs
        g = np.zeros((gs.np, 3))
        g[:, :gs.dim] = grad_du.detach().cpu().double().numpy()
        gE, gP, _ = gs.adjoint(dL_dx=g, want_E=True, want_phi=True)
        return (None, None, torch.from_numpy(gE).to(ctx.dev), torch.from_numpy(gP).to(ctx.dev))
