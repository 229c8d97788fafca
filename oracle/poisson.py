"""Geometric multigrid V-cycle for the Poisson equation on a uniform
periodic mesh (oracle side).

TEST INFRASTRUCTURE ONLY: used by tests/, never by the product library.

Sec. II.C names Enzo-P's `mg0` solver, a geometric multigrid V-cycle, the
solver of self-gravity in the paper's uniform-grid runs (Sec. III).  The
paper prints no formulas; the readings taken here are:

* Problem: lap(phi) = f on the cell centres of a uniform mesh (every leaf
  at one level, periodic on every axis), the 7-point Laplacian
  lap(phi)_c = (((((phi_{x-1} + phi_{x+1}) + phi_{y-1}) + phi_{y+1})
  + phi_{z-1}) + phi_{z+1} - 6 phi_c) / h^2.  The mean of f is removed
  first (a periodic problem is solvable only for zero-mean f) and the mean
  of phi is removed at the end (phi is defined up to a constant).
* Grids: the mesh's cells as one M^3 grid (M = root * 2^L * n per axis,
  cubic root arrays), coarsened by 2 while M is even and above 1.
* V-cycle on a grid of spacing h: two damped Jacobi sweeps (weight 6/7),
  phi <- (1 - w) phi + w ((sum of the 6 neighbours) - h^2 f) / 6; the
  residual r = f - lap(phi); restriction by the mean of the 8 children
  (summed in (dz, dy, dx) order, times 0.125); the coarse error from a
  V-cycle started at zero with spacing 2h; trilinear prolongation of the
  coarse error (weights 3/4 and 1/4 per axis towards the nearer coarse
  neighbour, along x, then y, then z) added to phi; two more Jacobi sweeps.
  A 1-cell grid returns 0; a grid of odd size above 1 is solved by 50
  Jacobi sweeps.
"""
from __future__ import annotations

import torch

OMEGA = 6.0 / 7.0
NU1 = NU2 = 2
COARSE_SWEEPS = 50


def _nb(phi):
    """(x-1, x+1, y-1, y+1, z-1, z+1) neighbours with periodic wrap; phi[z, y, x]."""
    return (torch.roll(phi, 1, 2), torch.roll(phi, -1, 2), torch.roll(phi, 1, 1), torch.roll(phi, -1, 1),
            torch.roll(phi, 1, 0), torch.roll(phi, -1, 0))


def _nbsum(phi):
    xm, xp, ym, yp, zm, zp = _nb(phi)
    return ((((xm + xp) + ym) + yp) + zm) + zp


def laplacian(phi, h):
    return (_nbsum(phi) - 6.0 * phi) / (h * h)


def jacobi(phi, f, h):
    return (1.0 - OMEGA) * phi + OMEGA * ((_nbsum(phi) - (h * h) * f) / 6.0)


def residual(phi, f, h):
    return f - laplacian(phi, h)


def restrict(r):
    M = r.shape[0] // 2
    v = r.view(M, 2, M, 2, M, 2)
    s = None
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                t = v[:, dz, :, dy, :, dx]
                s = t if s is None else s + t
    return s * 0.125


def prolong(ec):
    """Trilinear cell-centred interpolation of a coarse grid to twice its size."""
    M = ec.shape[0]
    out = torch.empty(2 * M, 2 * M, 2 * M, dtype=ec.dtype)
    for oz in range(2):
        sz = 1 if oz else -1
        for oy in range(2):
            sy = 1 if oy else -1
            for ox in range(2):
                sx = 1 if ox else -1

                def at(dz, dy, dx):
                    return torch.roll(ec, (-dz * sz, -dy * sy, -dx * sx), (0, 1, 2))
                c00 = 0.75 * at(0, 0, 0) + 0.25 * at(0, 0, 1)
                c10 = 0.75 * at(0, 1, 0) + 0.25 * at(0, 1, 1)
                c01 = 0.75 * at(1, 0, 0) + 0.25 * at(1, 0, 1)
                c11 = 0.75 * at(1, 1, 0) + 0.25 * at(1, 1, 1)
                c0 = 0.75 * c00 + 0.25 * c10
                c1 = 0.75 * c01 + 0.25 * c11
                out[oz::2, oy::2, ox::2] = 0.75 * c0 + 0.25 * c1
    return out


def vcycle(phi, f, h):
    M = phi.shape[0]
    if M == 1:
        return torch.zeros_like(phi)
    if M % 2 == 1:
        for _ in range(COARSE_SWEEPS):
            phi = jacobi(phi, f, h)
        return phi
    for _ in range(NU1):
        phi = jacobi(phi, f, h)
    fc = restrict(residual(phi, f, h))
    ec = vcycle(torch.zeros_like(fc), fc, 2.0 * h)
    phi = phi + prolong(ec)
    for _ in range(NU2):
        phi = jacobi(phi, f, h)
    return phi


def solve(f, h, cycles, inner="float64"):
    """V-cycles from phi = 0 on the mean-free f; returns (phi with zero
    mean, list of the residual max-norms after each cycle).  inner =
    "float32": mixed-precision defect correction, each cycle a float32
    V-cycle from zero on the float32-rounded float64 residual, its result
    added to the float64 phi (the attainable accuracy stays float64's: the
    residual that drives each cycle is computed in float64)."""
    f0 = f - f.mean()
    phi = torch.zeros_like(f0)
    norms = []
    for _ in range(cycles):
        if inner == "float64":
            phi = vcycle(phi, f0, h)
        else:
            r = residual(phi, f0, h).to(torch.float32)
            phi = phi + vcycle(torch.zeros_like(r), r, h).to(torch.float64)
        norms.append(float(residual(phi, f0, h).abs().max()))
    return phi - phi.mean(), norms


def to_global(mesh, V):
    """Leaf interiors V[B, n, n, n] of a uniform mesh as one grid [M, M, M]."""
    d = mesh.desc
    n = d.n
    L = int(mesh.leaves[0, 0])
    Mb = [r << L for r in d.root]
    G = torch.empty(Mb[2] * n, Mb[1] * n, Mb[0] * n, dtype=V.dtype)
    for b, (_, i, j, k) in enumerate(mesh.leaves):
        G[k * n:(k + 1) * n, j * n:(j + 1) * n, i * n:(i + 1) * n] = V[b]
    return G


def from_global(mesh, G):
    d = mesh.desc
    n = d.n
    out = torch.empty(mesh.n_leaves, n, n, n, dtype=G.dtype)
    for b, (_, i, j, k) in enumerate(mesh.leaves):
        out[b] = G[k * n:(k + 1) * n, j * n:(j + 1) * n, i * n:(i + 1) * n]
    return out
