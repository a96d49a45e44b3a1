"""``LiquidVolume``: the final liquid volume of a melting run as a differentiable function
of the per-node hot-wall temperature field and of the Stefan number.

Forward: a fresh lattice from the given initial enthalpy, the wall field on face
``face``, ``nsteps`` coupled steps with checkpoints every ``ckpt_every`` steps; returns
J = sum of f_l over the lattice.  Backward: the library's hand-written reverse sweep
(recompute each segment with its macroscopic tape, then the transposed step).  The
initial state is an input held fixed (it does not depend on the wall field, and on St
only through T(h0) of initially liquid nodes).
"""
from __future__ import annotations

import numpy as np
import torch

from .lbpc import LBPC


class LiquidVolume(torch.autograd.Function):
    @staticmethod
    def forward(ctx, T_wall, St, shape, params, h0, nsteps, ckpt_every, face=0):
        p = params.replace(St=float(St.item()))
        lat = LBPC(shape, p)
        lat.set_wall_temperature(face, T_wall.detach().double().cpu().numpy())
        lat.set_initial_h(np.asarray(h0, dtype=np.float64))
        J = lat.adjoint_forward(int(nsteps), int(ckpt_every))
        ctx.lat, ctx.face = lat, face
        ctx.tw_device, ctx.tw_dtype = T_wall.device, T_wall.dtype
        return torch.tensor(J, dtype=torch.float64, device=T_wall.device)

    @staticmethod
    def backward(ctx, gJ):
        g, dSt = ctx.lat.adjoint_backward(ctx.face)
        ctx.lat.release_adjoint_workspace()
        scale = float(gJ.item())
        gT = torch.from_numpy(g * scale).to(ctx.tw_device, ctx.tw_dtype)
        gSt = torch.tensor(dSt * scale, dtype=torch.float64, device=ctx.tw_device)
        return gT, gSt, None, None, None, None, None, None


def liquid_volume(T_wall, St, shape, params, h0, nsteps, ckpt_every, face=0):
    """J = sum f_l after nsteps; differentiable in T_wall (face-area tensor) and St."""
    return LiquidVolume.apply(T_wall, St, shape, params, h0, nsteps, ckpt_every, face)
