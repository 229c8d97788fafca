"""Tracer particles on the GPU against the oracle: leaf lookup bit-exact,
pushes bit-exact in float64 (positions and leaves, for float64 and float32
states), over several steps with migration between leaves, periodic wrap
and outflow loss.  Box extents 1.0 (block and cell widths powers of two:
the kernels scale by exact reciprocals) and 0.6 (they divide) both run."""
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
def test_push_bit_exact_over_steps(precision, extent):
    """Blob velocities with an ABC flow (ghosts refreshed by the oracle, then
    cast to the state precision): five pushes, positions and leaves equal
    bit for bit, many tracers crossing Block faces."""
    od, om, flags = _mesh(extent=extent)
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    U = OH.ghost_refresh(H.state(od, om.leaves, "blobs", count=12, seed=5, abc=0.3), om)
    dt = torch.float64 if precision == 8 else torch.float32
    Ud = U.to(dt).cuda().contiguous()
    Uo = U.to(dt)                       # the oracle reads the same values
    pos = _points(600, 2, extent)
    leaf = OP.locate(om, pos)
    pd = pos.cuda().contiguous()
    ld = leaf.to(torch.int32).cuda()
    dt_push = 0.12 * extent
    step = torch.full((1,), dt_push, dtype=torch.float64, device="cuda")
    moved = 0
    for _ in range(5):
        pos, leaf2 = OP.push(Uo, om, pos, leaf, dt_push)
        moved += int((leaf2 != leaf).sum())
        leaf = leaf2
        gm.particles_push(Ud, pd, ld, step)
        assert torch.equal(pd.cpu(), pos)
        assert torch.equal(ld.cpu().long(), leaf)
    assert moved > 20


def test_uniform_flow_wrap_and_outflow_loss():
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
