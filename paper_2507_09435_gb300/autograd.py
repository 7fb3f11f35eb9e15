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


class ImplicitSteps(torch.autograd.Function):
    """Several implicit load steps: ``ImplicitSteps.apply(gs, steps, E_p, phi_p)``
    commits ``steps`` one after the other from the scene's committed state
    and returns the final particle positions (np x dim).  The forward pass
    records each start-of-step state and converged increment; ``backward``
    runs the reverse chain (``mpm_adjoint_step``) from the last step to the
    first, restoring each recorded state, and leaves the scene at its final
    committed state."""

    @staticmethod
    def forward(ctx, gs, steps, E_p, phi_p):
        from . import mpm
        gs.set_params(E_p=E_p.detach().cpu().double().numpy(), phi_p=phi_p.detach().cpu().double().numpy())
        tape = []
        for st in steps:
            state = gs.particles(tau=False)
            gs.solve_staged(st)
            tape.append((state, gs.du()))
            gs.commit()
        final = gs.particles(tau=False)
        ctx.gs, ctx.steps, ctx.tape, ctx.final, ctx.dev = gs, steps, tape, final, E_p.device
        return torch.from_numpy(np.ascontiguousarray(final["x"][:, :gs.dim])).to(E_p.device)

    @staticmethod
    def backward(ctx, grad_x):
        from . import mpm
        gs = ctx.gs
        np_ = gs.np
        sbar = {"x": np.zeros((np_, 3)), "be": np.zeros((np_, 6)), "pc": np.zeros(np_), "F": np.zeros((np_, 3, 3))}
        sbar["x"][:, :gs.dim] = grad_x.detach().cpu().double().numpy()
        grads = {"E": np.zeros(np_), "phi": np.zeros(np_)}
        for st, (state, U) in zip(reversed(ctx.steps), reversed(ctx.tape)):
            mpm.mpm_set_state(gs.h, x=state["x"], be=state["be"], pc=state["pc"], F=state["F"])
            gs.begin(st)
            gs.set_du(U)
            mpm.mpm_adjoint_step(gs.h, np_, sbar, grads=grads)
        f = ctx.final
        mpm.mpm_set_state(gs.h, x=f["x"], be=f["be"], pc=f["pc"], F=f["F"])
        return (None, None, torch.from_numpy(grads["E"]).to(ctx.dev), torch.from_numpy(grads["phi"]).to(ctx.dev))
