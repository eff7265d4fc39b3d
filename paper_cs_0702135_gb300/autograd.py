"""torch.autograd.Function over the library's differentiable Hermite trajectory.

Argument marshalling only: the forward pass is nb_traj_forward (fixed shared
step, checkpoints on the device) and the backward pass nb_traj_backward
(recomputation per checkpoint segment, transposed corrector and predictor,
hand-written force VJP kernel).  Leaves are float64 tensors.
"""
from __future__ import annotations

import torch

from . import nb


class HermiteTrajectory(torch.autograd.Function):
    """(x0, v0, m) -> (x_T, v_T) after `steps` Hermite steps of 2^-level."""

    @staticmethod
    def forward(ctx, x0, v0, m, eps, level, steps, checkpoint_every, precision=nb.NB_DS):
        c = nb.Context(m.detach().cpu().numpy(), x0.detach().cpu().numpy(),
                       v0.detach().cpu().numpy(), float(eps), level_fixed=int(level),
                       precision=int(precision), flags=nb.NB_INIT_NO_FORCE)
        c.nb_traj_forward(int(steps), int(checkpoint_every))
        st = c.nb_get_state()
        ctx.nbctx = c
        ctx.device = x0.device
        return (torch.from_numpy(st["x"]).to(x0.device), torch.from_numpy(st["v"]).to(x0.device))

    @staticmethod
    def backward(ctx, gx, gv):
        xb, vb, mb = ctx.nbctx.nb_traj_backward(
            gx.detach().cpu().numpy() if gx is not None else torch.zeros(1).numpy(),
            gv.detach().cpu().numpy() if gv is not None else None)
        d = ctx.device
        return (torch.from_numpy(xb).to(d), torch.from_numpy(vb).to(d), torch.from_numpy(mb).to(d),
                None, None, None, None, None)


def hermite_trajectory(x0, v0, m, eps, level, steps, checkpoint_every, precision=nb.NB_DS):
    return HermiteTrajectory.apply(x0, v0, m, eps, level, steps, checkpoint_every, precision)
