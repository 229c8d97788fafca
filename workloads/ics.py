"""Seeded synthetic initial conditions for the hydro workloads.

This module is the one piece shared by the oracle and the CUDA path: it turns
a workload recipe (Sod tube, blob field, Sedov deposit, Gaussian random
field) into the initial conserved state on a given leaf list.  It holds none
of the method's arithmetic (no reconstruction, flux, refresh, flag or
reduction) and imports neither side.

Leaves are an int64 array [B, 4] of (level, i, j, k); the state is
U[B, 5, N, N, N] float64 (rho, rho*u, rho*v, rho*w, E), cells [z, y, x],
N = n + 2*ghosts, every cell (ghosts included) sampled at its centre
(with_internal_energy appends rho*e for the dual-energy formalism).
"""
from __future__ import annotations

import numpy as np
import torch


def cell_centres(leaves, root, n, ghosts, lo, hi, device="cpu"):
    """x, y, z cell-centre coordinates, each [B, N, N, N] float64."""
    leaves = torch.as_tensor(np.asarray(leaves), dtype=torch.int64, device=device)
    N = n + 2 * ghosts
    L = leaves[:, 0].to(torch.float64)
    out = []
    for a in range(3):
        ext = (hi[a] - lo[a]) / root[a]              # root block width
        bw = ext / torch.pow(2.0, L)                 # block width per leaf
        dx = bw / n
        idx = torch.arange(N, dtype=torch.float64, device=device) - ghosts + 0.5
        c = lo[a] + leaves[:, 1 + a].to(torch.float64) * bw
        out.append(c.view(-1, 1) + dx.view(-1, 1) * idx.view(1, -1))
    B = leaves.shape[0]
    x = out[0].view(B, 1, 1, N).expand(B, N, N, N)
    y = out[1].view(B, 1, N, 1).expand(B, N, N, N)
    z = out[2].view(B, N, 1, 1).expand(B, N, N, N)
    return x, y, z


def conserved(rho, u, v, w, p, gamma):
    """Initial conserved state from primitive fields (ideal gas)."""
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, rho * u, rho * v, rho * w, E], 1)


def with_internal_energy(U):
    """The state with a sixth field, the internal energy density
    rho e = E - |m|^2 / (2 rho), for runs with the dual-energy formalism."""
    ke = 0.5 * (U[:, 1] * U[:, 1] + U[:, 2] * U[:, 2] + U[:, 3] * U[:, 3]) / U[:, 0]
    return torch.cat([U, (U[:, 4] - ke).unsqueeze(1)], 1)


def sod(leaves, root, n, ghosts, lo, hi, gamma, x0=0.5, axis=0, device="cpu"):
    """Sod shock tube along an axis: (rho, p) = (1, 1) below x0 and
    (0.125, 0.1) above, at rest."""
    c = cell_centres(leaves, root, n, ghosts, lo, hi, device)[axis]
    left = c < x0
    one = torch.ones(c.shape, dtype=torch.float64, device=c.device)
    rho = torch.where(left, one, 0.125 * one)
    p = torch.where(left, one, 0.1 * one)
    z = torch.zeros_like(rho)
    return conserved(rho, z, z, z, p, gamma)


def uniform(leaves, root, n, ghosts, lo, hi, gamma, rho=1.0, vel=(0.0, 0.0, 0.0), p=1.0, device="cpu"):
    x = cell_centres(leaves, root, n, ghosts, lo, hi, device)[0]
    one = torch.ones_like(x)
    return conserved(rho * one, vel[0] * one, vel[1] * one, vel[2] * one, p * one, gamma)


def blob_params(count, seed):
    """Blob centres ~U[0,1)^3, radii ~U[0.02, 0.05), velocities ~N(0, 0.1^2)
    per component, drawn in that order from numpy's PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.random((count, 3))
    radii = rng.uniform(0.02, 0.05, count)
    vel = rng.normal(0.0, 0.1, (count, 3))
    return centres, radii, vel


def blobs(leaves, root, n, ghosts, lo, hi, gamma, count=64, seed=0, contrast=10.0, p0=1.0,
          device="cpu", chunk=64, abc=0.0):
    """Blob field in a periodic unit box: ambient rho=1 at rest; inside a blob
    (periodic minimum-image distance below its radius) rho=contrast and the
    blob's velocity; overlaps go to the lowest blob index; p = p0.  With
    abc > 0 an Arnold-Beltrami-Childress flow of amplitude abc (A = B = C,
    wavenumber 2 pi) is added to every cell's velocity, so that no region is
    at rest."""
    centres, radii, vel = blob_params(count, seed)
    leaves_np = np.asarray(leaves, dtype=np.int64)
    B = leaves_np.shape[0]
    N = n + 2 * ghosts
    box = np.array([hi[a] - lo[a] for a in range(3)])
    # leaf boxes (with the ghost margin) for the pair test
    L = leaves_np[:, 0].astype(np.float64)
    bw = np.stack([(box[a] / root[a]) / 2.0 ** L for a in range(3)], 1)
    blo = np.stack([lo[a] + leaves_np[:, 1 + a] * bw[:, a] for a in range(3)], 1)
    margin = bw * ghosts / n
    c0 = (blo - margin)[:, None, :]
    c1 = (blo + bw + margin)[:, None, :]
    cen = centres[None, :, :] * box
    d = np.maximum(np.maximum(c0 - cen, cen - c1), 0.0)
    # periodic images: distance to the box through the wrap
    dw = np.minimum(d, np.maximum(np.maximum(c0 - (cen + box), (cen + box) - c1), 0.0))
    dw = np.minimum(dw, np.maximum(np.maximum(c0 - (cen - box), (cen - box) - c1), 0.0))
    hit = (dw * dw).sum(-1) < (radii[None, :] ** 2)
    pb, pi = np.nonzero(hit)
    owner = torch.full((B, N * N * N), count, dtype=torch.int64, device=device)
    if len(pb):
        x, y, z = cell_centres(leaves_np, root, n, ghosts, lo, hi, device)
        xyz = torch.stack([x.reshape(B, -1), y.reshape(B, -1), z.reshape(B, -1)], 1)  # [B, 3, N^3]
        cen_t = torch.as_tensor(centres * box, device=device)
        rad_t = torch.as_tensor(radii, device=device)
        box_t = torch.as_tensor(box, device=device).view(1, 3, 1)
        pb_t = torch.as_tensor(pb, device=device)
        pi_t = torch.as_tensor(pi, device=device)
        for s in range(0, len(pb), chunk):
            b, i = pb_t[s:s + chunk], pi_t[s:s + chunk]
            dd = xyz[b] - cen_t[i].view(-1, 3, 1)
            dd = dd - box_t * torch.round(dd / box_t)
            inside = (dd * dd).sum(1) < (rad_t[i] ** 2).view(-1, 1)
            cand = torch.where(inside, i.view(-1, 1), torch.full_like(inside, count, dtype=torch.int64))
            owner.scatter_reduce_(0, b.view(-1, 1).expand_as(cand), cand, reduce="amin")
    owner = owner.view(B, N, N, N)
    inside = owner < count
    vel_t = torch.cat([torch.as_tensor(vel, device=device), torch.zeros(1, 3, dtype=torch.float64, device=device)])
    v = vel_t[owner]
    one = torch.ones(inside.shape, dtype=torch.float64, device=inside.device)
    rho = torch.where(inside, contrast * one, one)
    p = torch.full_like(rho, p0)
    vx, vy, vz = v[..., 0], v[..., 1], v[..., 2]
    if abc > 0.0:
        x, y, z = cell_centres(leaves_np, root, n, ghosts, lo, hi, device)
        k = 2.0 * np.pi
        vx = vx + abc * (torch.sin(k * z) + torch.cos(k * y))
        vy = vy + abc * (torch.sin(k * x) + torch.cos(k * z))
        vz = vz + abc * (torch.sin(k * y) + torch.cos(k * x))
    return conserved(rho, vx, vy, vz, p, gamma)


def sedov(leaves, root, n, ghosts, lo, hi, gamma, E=1.0, rho0=1.0, p0=1e-5, half_width=None,
          max_level=5, device="cpu"):
    """Sedov deposit: energy E spread uniformly over the cube of half-width
    half_width (default: one cell at max_level) centred in the box; each cell
    receives E times its overlap fraction with the cube, so the deposit is
    conservative at every level.  rho = rho0, p = p0 elsewhere."""
    x, y, z = cell_centres(leaves, root, n, ghosts, lo, hi, device)
    leaves_t = torch.as_tensor(np.asarray(leaves), dtype=torch.int64, device=device)
    dxl = ((hi[0] - lo[0]) / root[0] / n) / torch.pow(2.0, leaves_t[:, 0].to(torch.float64))
    if half_width is None:
        half_width = (hi[0] - lo[0]) / root[0] / n / 2.0 ** max_level
    h = dxl.view(-1, 1, 1, 1)
    frac = torch.ones_like(x)
    for a, c in enumerate((x, y, z)):
        mid = 0.5 * (lo[a] + hi[a])
        ov = torch.clamp(torch.minimum(c + 0.5 * h, torch.full_like(c, mid + half_width))
                         - torch.maximum(c - 0.5 * h, torch.full_like(c, mid - half_width)), min=0.0)
        frac = frac * ov
    frac = frac / (2.0 * half_width) ** 3
    rho = torch.full_like(x, rho0)
    zz = torch.zeros_like(x)
    U = conserved(rho, zz, zz, zz, torch.full_like(x, p0), gamma)
    U[:, 4] = U[:, 4] + E * frac / (h * h * h)
    return U


def grf_density(N, seed, amp=0.1, slope=-2.0):
    """1 + amp*delta on an N^3 periodic grid: real white noise (PCG64(seed)),
    shaped in Fourier space by sqrt(P(k)) with P ~ k^slope, k = 0 removed,
    normalised to unit standard deviation.  Returned [z, y, x] float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.normal(size=(N, N, N))
    F = np.fft.rfftn(white)
    kz = np.fft.fftfreq(N) * N
    ky = np.fft.fftfreq(N) * N
    kx = np.fft.rfftfreq(N) * N
    k = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
    shape = np.zeros_like(k)
    nz = k > 0
    shape[nz] = k[nz] ** (slope / 2.0)
    delta = np.fft.irfftn(F * shape, s=(N, N, N), axes=(0, 1, 2))
    delta = (delta - delta.mean()) / delta.std()
    return 1.0 + amp * delta


def grf(leaves, root, n, ghosts, gamma, seed=0, amp=0.1, p0=1.0, device="cpu"):
    """Gaussian-random-field density on a single-level periodic mesh, p = p0,
    at rest.  Ghost cells take the periodic image."""
    leaves = np.asarray(leaves, dtype=np.int64)
    assert (leaves[:, 0] == 0).all()
    Ng = root[0] * n
    assert root[0] == root[1] == root[2]
    rho_grid = torch.as_tensor(grf_density(Ng, seed, amp), device=device)
    N = n + 2 * ghosts
    ar = torch.arange(N, device=device) - ghosts
    B = len(leaves)
    rho = torch.empty((B, N, N, N), dtype=torch.float64, device=device)
    for b, (_, i, j, k) in enumerate(leaves):
        xi = (i * n + ar) % Ng
        yi = (j * n + ar) % Ng
        zi = (k * n + ar) % Ng
        rho[b] = rho_grid[zi][:, yi][:, :, xi]
    z = torch.zeros_like(rho)
    return conserved(rho, z, z, z, torch.full_like(rho, p0), gamma)
