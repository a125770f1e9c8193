"""torch.autograd face of avl_adjoint: the field energy J = 1/2 sum E(T)^2 dx
as a differentiable function of the mode amplitudes and beam x-drifts of one
species' initial distribution.  Forward and gradient both come from one
avl_adjoint call (forward run, checkpointed backward run on the GPU); the
backward hook only scales the stored gradient by the incoming one."""
from __future__ import annotations

import torch

from . import avl as A


def _theta(template, amps, drifts):
    beams = []
    for b, (n, u, vth) in enumerate(template["beams"]):
        u = list(u) + [0.0] * (3 - len(u))
        u[0] = float(drifts[b])
        beams.append((n, tuple(u), vth))
    modes = [(m, float(amps[k]), ph) for k, (m, _, ph) in enumerate(template["modes"])]
    return A.make_f0(beams, modes)


class FieldEnergy(torch.autograd.Function):
    """J = FieldEnergy.apply(amps, drifts, sim, s, template, nsteps, ckpt_every)

    amps: (nmode,) float64 tensor, drifts: (nbeam,) float64 tensor (x-drift
    of each beam); template: {"beams": [(n, u, vth)], "modes": [(mode, amp,
    phase)]} giving everything else of f0.  Returns a 0-d float64 tensor."""

    @staticmethod
    def forward(ctx, amps, drifts, sim, s, template, nsteps, ckpt_every):
        theta = _theta(template, amps.detach().cpu().tolist(), drifts.detach().cpu().tolist())
        J, g_amp, g_u = sim.adjoint(s, theta, nsteps, ckpt_every)
        ctx.save_for_backward(torch.as_tensor(g_amp, dtype=amps.dtype, device=amps.device),
                              torch.as_tensor(g_u, dtype=drifts.dtype, device=drifts.device))
        return torch.tensor(J, dtype=torch.float64, device=amps.device)

    @staticmethod
    def backward(ctx, grad_out):
        g_amp, g_u = ctx.saved_tensors
        return grad_out * g_amp, grad_out * g_u, None, None, None, None, None
