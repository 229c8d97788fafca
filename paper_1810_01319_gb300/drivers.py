"""Run drivers over the C ABI: mesh adaptation (refresh, refinement flags,
octree rebuild, remap) and an adaptive time loop.  Every numerical step runs
in the library's kernels; this module only sequences the calls."""
from __future__ import annotations

import numpy as np
import torch

from . import Mesh


def may_change(leaves, flags) -> bool:
    """False when the flags cannot change the mesh: no leaf asks for
    refinement and no parent has all eight children flagged for coarsening
    (a coarsening needs the whole octet).  Then the rebuild can be skipped."""
    if (flags > 0).any():
        return True
    c = (flags < 0) & (leaves[:, 0] > 0)
    if not c.any():
        return False
    lv = leaves[c].astype(np.int64)
    parents = np.stack([lv[:, 0] - 1, lv[:, 1] >> 1, lv[:, 2] >> 1, lv[:, 3] >> 1], axis=1)
    _, counts = np.unique(parents, axis=0, return_counts=True)
    return bool((counts == 8).any())


def adapt(mesh: Mesh, U, field: int = 0, tau: float = 0.3, tau_c: float | None = None, allow_coarsen=True):
    """One adaptation (Sec. II.B, Refine with Prolong/Restrict): returns the
    (possibly new) mesh and state.  U's ghosts are refreshed in place."""
    tau_c = tau / 4 if tau_c is None else tau_c
    mesh.ghost_refresh(U)
    flags = mesh.refine_flags(U, field, tau, tau_c).cpu().numpy()
    if not allow_coarsen:
        flags = np.where(flags > 0, 1, 0).astype(np.int8)
    if not may_change(mesh.leaves, flags):
        return mesh, U
    new = Mesh(mesh.desc, mesh, flags)
    if new.n_leaves == mesh.n_leaves and np.array_equal(new.leaves, mesh.leaves):
        return mesh, U
    return new, new.remap_from(mesh, U)


def run_adaptive(mesh: Mesh, U, t_end: float, cfl: float = 0.4, field: int = 0, tau: float = 0.3,
                 adapt_every: int = 1, max_steps: int = 100000, dts=None, callback=None):
    """Advance to t_end (or through a given dt sequence), adapting every
    `adapt_every` steps before the step.  Returns (mesh, U, t, steps)."""
    dt = torch.zeros(1, dtype=torch.float64, device=U.device)
    t, s = 0.0, 0
    while s < max_steps and (dts is None and t < t_end or dts is not None and s < len(dts)):
        if s % adapt_every == 0:
            mesh, U = adapt(mesh, U, field, tau)
        if dts is not None:
            dt.fill_(float(dts[s]))
        else:
            mesh.reduce(U, cfl, dt_next=dt)
            d = float(dt)
            if t + d > t_end:
                dt.fill_(t_end - t)
        mesh.hydro_step(U, dt, s, cfl)
        t += float(dt)
        s += 1
        if callback:
            callback(mesh, U, t, s)
    return mesh, U, t, s
