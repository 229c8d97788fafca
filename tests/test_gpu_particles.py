"""Tracer particles on the GPU against the oracle.

Leaf lookup is integer work on identical float64 positions: bit-exact.

A push is compared with the oracle's plain definition (velocity = momentum
divided by floored density, one float64 division per cell and component).
The kernel forms 1/rho as a float32 seed refined by two float64 Newton
steps and multiplies, which stays within a few ulp of the quotient, so
pushes are compared at a tolerance derived from that arithmetic:

* per corner cell, the kernel's velocity and the oracle's quotient differ
  by at most 6 u |v| (u = 2^-53: at most 2 ulp in the reciprocal, one
  rounding of the product, one rounding of the quotient);
* the trilinear interpolation (seven non-negative-weight lerps, three
  levels deep, the same operations on both sides) adds at most 18 u vmax
  of rounding on each side, so the interpolated velocities differ by at
  most 32 u vmax = 2^-48 vmax, vmax the largest |velocity| of the state;
* the new position x + dt v (and its periodic wrap) adds up to one ulp of
  the extent for each rounding that may fall differently: two.

Hence, from identical inputs, |x_gpu - x_oracle| <= dt 2^-48 vmax +
2^-51 extent per push and axis.  The new leaf must be the oracle's leaf
except for tracers whose oracle position lies within that bound of a
block face at max_level (where floor((x - lo) / w) may fall either way);
there the GPU's leaf must contain the GPU's own position.  A chain of five
pushes is checked at five times the bound, the velocity's Lipschitz
growth over five short pushes being far below the factor.  Box extents
1.0 (block and cell widths powers of two: the kernels scale by exact
reciprocals) and 0.6 (they divide) both run."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM
from oracle import particles as OP

pytestmark = pytest.mark.gpu


EXTENTS = [1.0, 0.6]


def _mesh(bc=(OM.PERIODIC,) * 3, extent=1.0):
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=2, bc=bc, hi=(extent,) * 3)
    om, flags = H.ic_refined(od, "blobs", count=12, seed=5)
    assert om.leaves[:, 0].max() == 2
    return od, om, flags


def _points(n, seed, extent=1.0):
    g = torch.Generator().manual_seed(seed)
    return torch.rand(3, n, generator=g, dtype=torch.float64) * extent


def _vmax(U):
    rho = U[:, 0].double().clamp_min(OP.RHO_FLOOR)
    return max(float((U[:, 1 + c].double() / rho).abs().max()) for c in range(3))


def _bound(dt, vmax, extent):
    return dt * vmax * 2.0 ** -48 + extent * 2.0 ** -51


def _near_face(od, pos, tol):
    """Tracers within tol of a block face at max_level on any axis."""
    w = (od.hi[0] - od.lo[0]) / od.root[0] / (1 << od.max_level)
    near = torch.zeros(pos.shape[1], dtype=torch.bool)
    for a in range(3):
        s = (pos[a] - od.lo[a]) / w
        near |= (s - torch.round(s)).abs() * w <= tol
    return near


def _check_push(od, om, pos_g, leaf_g, pos_o, leaf_o, tol):
    err = float((pos_g - pos_o).abs().max()) if pos_o.numel() else 0.0
    assert err <= tol, f"position differs by {err:.3e} > {tol:.3e}"
    assert torch.equal(leaf_g < 0, leaf_o < 0)
    differ = (leaf_g != leaf_o) & (leaf_o >= 0)
    if differ.any():
        near = _near_face(od, pos_o, tol)
        assert bool(near[differ].all()), "a leaf differs away from a block face"
        idx = torch.nonzero(differ).flatten()
        assert torch.equal(leaf_g[idx], OP.locate(om, pos_g[:, idx]))
    return int(differ.sum())


@pytest.mark.parametrize("extent", EXTENTS)
def test_locate_bit_exact(extent):
    od, om, flags = _mesh(extent=extent)
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    pos = _points(3000, 1, extent)
    pos[:, :8] = torch.tensor([[0.0, 0.25, 0.5, 0.125, 0.999999, 0.0625, 0.75, 0.375]] * 3,
                              dtype=torch.float64) * extent
    leaf = gm.particles_locate(pos.cuda().contiguous())
    assert torch.equal(leaf.cpu().long(), OP.locate(om, pos))


@pytest.mark.parametrize("extent", EXTENTS)
@pytest.mark.parametrize("precision", [8, 4])
def test_push_matches_oracle(precision, extent):
    """Blob velocities with an ABC flow (ghosts refreshed by the oracle, then
    cast to the state precision).  Each push starts from the oracle's
    positions and leaves and must land within the per-push bound; then a
    chain of five pushes on the GPU's own positions stays within five times
    the bound.  Many tracers cross Block faces."""
    od, om, flags = _mesh(extent=extent)
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    U = OH.ghost_refresh(H.state(od, om.leaves, "blobs", count=12, seed=5, abc=0.3), om)
    dty = torch.float64 if precision == 8 else torch.float32
    Ud = U.to(dty).cuda().contiguous()
    Uo = U.to(dty)                       # the oracle reads the same values
    vmax = _vmax(Uo)
    pos = _points(600, 2, extent)
    leaf = OP.locate(om, pos)
    dt_push = 0.12 * extent
    tol = _bound(dt_push, vmax, extent)
    step = torch.full((1,), dt_push, dtype=torch.float64, device="cuda")
    # one push at a time from the oracle's state of the tracers
    moved = 0
    for _ in range(5):
        pd = pos.cuda().contiguous()
        ld = leaf.to(torch.int32).cuda()
        pos2, leaf2 = OP.push(Uo, om, pos, leaf, dt_push)
        gm.particles_push(Ud, pd, ld, step)
        _check_push(od, om, pd.cpu(), ld.cpu().long(), pos2, leaf2, tol)
        moved += int((leaf2 != leaf).sum())
        pos, leaf = pos2, leaf2
    assert moved > 20
    # a chain of five pushes on the GPU's own positions
    pos = _points(600, 2, extent)
    leaf = OP.locate(om, pos)
    pd, ld = pos.cuda().contiguous(), leaf.to(torch.int32).cuda()
    for k in range(5):
        pos, leaf = OP.push(Uo, om, pos, leaf, dt_push)
        gm.particles_push(Ud, pd, ld, step)
        _check_push(od, om, pd.cpu(), ld.cpu().long(), pos, leaf, (k + 1) * tol)


def test_uniform_flow_wrap_and_outflow_loss():
    """Uniform velocity: every corner quotient m / rho with rho = 1 is exact
    on both sides, so positions and leaves agree bit for bit."""
    od, om, flags = _mesh(bc=(OM.OUTFLOW, OM.PERIODIC, OM.PERIODIC))
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    from workloads import ics
    x, _, _ = ics.cell_centres(om.leaves, od.root, od.n, od.ghosts, od.lo, od.hi)
    one = torch.ones_like(x)
    U = ics.conserved(one, 0.4 * one, -0.7 * one, 0.3 * one, one, od.gamma)
    pos = _points(800, 3)
    leaf = OP.locate(om, pos)
    pd, ld = pos.cuda().contiguous(), leaf.to(torch.int32).cuda()
    step = torch.full((1,), 0.2, dtype=torch.float64, device="cuda")
    for _ in range(3):
        pos, leaf = OP.push(U, om, pos, leaf, 0.2)
        gm.particles_push(U.cuda().contiguous(), pd, ld, step)
    assert torch.equal(pd.cpu(), pos) and torch.equal(ld.cpu().long(), leaf)
    lost = int((leaf < 0).sum())
    assert 0 < lost < 800
