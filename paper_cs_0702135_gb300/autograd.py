"""torch.autograd.Function over the library's differentiable Hermite trajectory.

Argument marshalling only: the forward pass is nb_init_dev + nb_traj_forward
(fixed shared step, checkpoints on the device) + nb_get_state_dev, the backward
pass nb_traj_backward_dev (recomputation per checkpoint segment, transposed
corrector and predictor, hand-written force VJP kernel).  Leaves are float64
CUDA tensors; state, cotangents and gradients stay on the device, and the
library runs on the leaves' current torch stream.  The library context lives
from the forward pass to the end of the backward pass (or until the graph is
freed), so a second backward through the same trajectory is refused.
"""
from __future__ import annotations

import torch

from . import nb


class HermiteTrajectory(torch.autograd.Function):
    """(x0, v0, m) -> (x_T, v_T) after `steps` Hermite steps of 2^-level."""

    @staticmethod
    def forward(ctx, x0, v0, m, eps, level, steps, checkpoint_every, precision=nb.NB_DS):
        if x0.device.type != "cuda":
            raise ValueError("hermite_trajectory needs CUDA tensors")
        stream = torch.cuda.current_stream(x0.device).cuda_stream
        xc, vc, mc = (t.detach().to(torch.float64).contiguous() for t in (x0, v0, m))
        c = nb.Context.from_device(mc, xc, vc, float(eps), level_fixed=int(level),
                                   precision=int(precision), flags=nb.NB_INIT_NO_FORCE, stream=stream)
        try:
            c.nb_traj_forward(int(steps), int(checkpoint_every))
            xT, vT = torch.empty_like(xc), torch.empty_like(vc)
            c.nb_get_state_dev(d_x=xT, d_v=vT)
        except Exception:
            c.nb_free()
            raise
        ctx.nbctx = c
        return xT, vT

    @staticmethod
    def backward(ctx, gx, gv):
        c = ctx.nbctx
        if c is None:
            raise RuntimeError("hermite_trajectory: the trajectory was already differentiated once")
        ctx.nbctx = None
        try:
            n = c.n
            dev = gx.device if gx is not None else gv.device
            z = torch.zeros((n, 3), dtype=torch.float64, device=dev)
            gxc = z if gx is None else gx.to(torch.float64).contiguous()
            gvc = None if gv is None else gv.to(torch.float64).contiguous()
            xb, vb = torch.empty_like(z), torch.empty_like(z)
            mb = torch.empty(n, dtype=torch.float64, device=dev)
            c.nb_traj_backward_dev(gxc, gvc, xb, vb, mb)
        finally:
            c.nb_free()
        return xb, vb, mb, None, None, None, None, None


def hermite_trajectory(x0, v0, m, eps, level, steps, checkpoint_every, precision=nb.NB_DS):
    return HermiteTrajectory.apply(x0, v0, m, eps, level, steps, checkpoint_every, precision)
