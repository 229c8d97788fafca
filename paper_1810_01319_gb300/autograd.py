"""Differentiable rollout of the hydro step: gradients of a loss on the
final state with respect to the initial state, through the library's
hand-written adjoint (cello_hydro_adjoint_step), dt held fixed, with
checkpoints every k steps and recomputation inside each segment."""
from __future__ import annotations

import torch


class HydroRollout(torch.autograd.Function):
    """U_final = step_{n-1} o ... o step_0 (U0) on a fixed mesh (any levels and
    boundaries; the mesh is not adapted inside the rollout)."""

    @staticmethod
    def forward(ctx, U0, mesh, dts, cycle0, every):
        U = U0.detach().clone().contiguous()
        dt = torch.empty(1, dtype=torch.float64, device=U.device)
        ckpt = {}
        for s, v in enumerate(dts):
            if s % every == 0:
                ckpt[s] = U.clone()
            dt.fill_(float(v))
            mesh.hydro_step(U, dt, cycle0 + s)
        ctx.mesh, ctx.dts, ctx.cycle0, ctx.every, ctx.ckpt = mesh, [float(v) for v in dts], cycle0, every, ckpt
        return U

    @staticmethod
    def backward(ctx, gU):
        mesh, dts, cycle0, every = ctx.mesh, ctx.dts, ctx.cycle0, ctx.every
        lam = gU.detach().clone().contiguous()
        dt = torch.empty(1, dtype=torch.float64, device=lam.device)
        n = len(dts)
        for s0 in sorted(ctx.ckpt, reverse=True):
            s1 = min(s0 + every, n)
            U = ctx.ckpt[s0].clone()
            states = [ctx.ckpt[s0]]
            for s in range(s0, s1 - 1):               # recompute the segment's start states
                dt.fill_(dts[s])
                mesh.hydro_step(U, dt, cycle0 + s)
                states.append(U.clone())
            for s in range(s1 - 1, s0 - 1, -1):
                dt.fill_(dts[s])
                mesh.hydro_adjoint_step(states[s - s0], lam, dt, cycle0 + s)
        ctx.ckpt = None
        return lam, None, None, None, None


def rollout(mesh, U0, dts, cycle0: int = 0, checkpoint_every: int = 10):
    """Advance U0 by len(dts) steps with the given dt sequence; differentiable
    with respect to U0."""
    return HydroRollout.apply(U0, mesh, list(dts), int(cycle0), int(checkpoint_every))
