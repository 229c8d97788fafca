"""Tracer particles on the array-of-octrees mesh (oracle side).

TEST INFRASTRUCTURE ONLY: used by tests/, never by the product library.

The paper's Cello supports Lagrangian particles next to the grid fields:
particles move between Blocks (Sec. II.B, Fig. 4), and the hydro scaling
workload of Sec. III carries tracer particles.  The paper prints no particle
formulas; the readings taken here are:

* A tracer is a position (x, y, z) in float64 and the index of the leaf that
  contains it.  The containing leaf of a point is found from the block index
  of the point at max_level, b_a = floor((x_a - lo_a) / w) with w the block
  width at max_level (clamped into the root array), whose Morton key (the
  key of mesh.py) lies in [key(leaf), key(leaf) + 8^(max_level - L)) for
  exactly one leaf: the last leaf in key order whose key does not exceed it.
* The tracer velocity is the fluid velocity, momentum divided by density
  (the density floored at 1e-10 as in the primitives of the sweep), one
  float64 division per cell and component, interpolated trilinearly
  between the cell centres of the containing leaf's padded block (its ghost
  layer refreshed), linear along x, then y, then z.
* One step moves every live tracer by dt times that velocity (forward
  Euler), wraps it into the box along periodic axes and marks it lost
  (leaf -1; a lost tracer is not moved again) when it leaves through an
  outflow face, then locates it again: a tracer that crossed a Block face
  migrates to its new leaf.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .mesh import PERIODIC, Mesh, morton_key

RHO_FLOOR = 1e-10


def block_width(mesh: Mesh):
    d = mesh.desc
    return (d.hi[0] - d.lo[0]) / d.root[0] / (1 << d.max_level)


def locate(mesh: Mesh, pos):
    """Leaf index of each point (pos [3, P] float64 tensor), by the Morton
    key of its block at max_level."""
    d = mesh.desc
    w = block_width(mesh)
    keys = np.array([morton_key(d, *map(int, lf)) for lf in mesh.leaves], dtype=np.int64)
    out = np.empty(pos.shape[1], dtype=np.int64)
    for p in range(pos.shape[1]):
        b = []
        for a in range(3):
            nb = d.root[a] << d.max_level
            v = math.floor((float(pos[a, p]) - d.lo[a]) / w)
            b.append(min(max(v, 0), nb - 1))
        k = morton_key(d, d.max_level, *b)
        out[p] = int(np.searchsorted(keys, k, side="right")) - 1
    return torch.from_numpy(out)


def velocity(U, mesh: Mesh, pos, leaf):
    """Trilinear interpolation of the cell-centred velocity (u, v, w) at each
    point from its leaf's padded block; returns [3, P] float64."""
    d = mesh.desc
    n, g = d.n, d.ghosts
    out = torch.zeros(3, pos.shape[1], dtype=torch.float64)
    for p in range(pos.shape[1]):
        b = int(leaf[p])
        L, li, lj, lk = (int(v) for v in mesh.leaves[b])
        dx = d.dx(L)
        i0, f = [], []
        for a, lidx in enumerate((li, lj, lk)):
            s = (float(pos[a, p]) - (d.lo[a] + (lidx * n) * dx)) / dx - 0.5
            c = math.floor(s)
            i0.append(c + g)
            f.append(s - c)
        for comp in range(3):
            def vel(z, y, x):
                rho = max(float(U[b, 0, z, y, x]), RHO_FLOOR)
                return float(U[b, 1 + comp, z, y, x]) / rho
            x0, y0, z0 = i0
            fx, fy, fz = f
            c00 = vel(z0, y0, x0) * (1.0 - fx) + vel(z0, y0, x0 + 1) * fx
            c10 = vel(z0, y0 + 1, x0) * (1.0 - fx) + vel(z0, y0 + 1, x0 + 1) * fx
            c01 = vel(z0 + 1, y0, x0) * (1.0 - fx) + vel(z0 + 1, y0, x0 + 1) * fx
            c11 = vel(z0 + 1, y0 + 1, x0) * (1.0 - fx) + vel(z0 + 1, y0 + 1, x0 + 1) * fx
            c0 = c00 * (1.0 - fy) + c10 * fy
            c1 = c01 * (1.0 - fy) + c11 * fy
            out[comp, p] = c0 * (1.0 - fz) + c1 * fz
    return out


def push(U, mesh: Mesh, pos, leaf, dt: float):
    """One tracer step (see the module docstring); returns (pos, leaf)."""
    d = mesh.desc
    pos = pos.clone()
    leaf = leaf.clone()
    live = leaf >= 0
    idx = torch.nonzero(live).flatten()
    if len(idx) == 0:
        return pos, leaf
    vel = velocity(U, mesh, pos[:, idx], leaf[idx])
    for a in range(3):
        x = pos[a, idx] + dt * vel[a]
        ext = d.hi[a] - d.lo[a]
        if d.bc[a] == PERIODIC:
            x = torch.where(x < d.lo[a], x + ext, torch.where(x >= d.hi[a], x - ext, x))
        else:
            out = (x < d.lo[a]) | (x >= d.hi[a])
            leaf[idx[out]] = -1
        pos[a, idx] = x
    keep = leaf[idx] >= 0
    if keep.any():
        k = idx[keep]
        leaf[k] = locate(mesh, pos[:, k])
    return pos, leaf
