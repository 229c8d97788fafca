"""GPU parity of the integer octree, the neighbour table and the refinement
flags against the oracle: bit-exact."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,bc,root,lmax", [
    (0, (OM.PERIODIC,) * 3, (2, 2, 2), 2),
    (1, (OM.OUTFLOW, OM.PERIODIC, OM.PERIODIC), (3, 2, 1), 3),
    (2, (OM.OUTFLOW,) * 3, (1, 1, 1), 3),
    (3, (OM.PERIODIC, OM.OUTFLOW, OM.PERIODIC), (2, 1, 2), 2),
])
def test_octree_and_neighbour_table_bit_exact(seed, bc, root, lmax):
    od = H.oracle_desc(root=root, n=8, lmax=lmax, bc=bc)
    meshes, flags = H.flag_sequence(od, rounds=lmax + 1, seed=seed, p_refine=0.35, p_coarsen=0.25)
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    om = meshes[-1]
    assert np.array_equal(gm.leaves.astype(np.int64), om.leaves)
    k1, i1, f1 = gm.neighbour_table()
    k2, i2, f2 = OM.neighbour_table(om)
    assert np.array_equal(k1, k2) and np.array_equal(i1, i2) and np.array_equal(f1, f2)


def test_root_mesh_large():
    od = H.oracle_desc(root=(16, 16, 16), n=32, lmax=2)
    gm = H.gpu_mesh_from_flags(od, [], 4)
    om = OM.root_mesh(od)
    assert np.array_equal(gm.leaves.astype(np.int64), om.leaves)
    k1, i1, _ = gm.neighbour_table()
    k2, i2, _ = OM.neighbour_table(om)
    assert np.array_equal(k1, k2) and np.array_equal(i1, i2)


@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("field", [0, 4])
def test_refine_flags_bit_exact(precision, field):
    od = H.oracle_desc(root=(2, 2, 1), n=16, lmax=2, bc=(OM.PERIODIC, OM.PERIODIC, OM.OUTFLOW))
    om, flags = H.ic_refined(od, "blobs", count=16, seed=4)
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    U0 = H.state(od, om.leaves, "blobs", count=16, seed=4)
    # pressure jumps large enough to flag some leaves on the pressure criterion
    U0[:, 4] *= 1.0 + 0.8 * (torch.rand(U0[:, 4].shape, generator=torch.Generator().manual_seed(1),
                                        dtype=torch.float64) > 0.999)
    Ug = U0.to(gm.dtype).cuda().contiguous()
    gm.ghost_refresh(Ug)
    fg = gm.refine_flags(Ug, field, 0.3, 0.075).cpu().numpy()
    Uo = OH.ghost_refresh(U0.to(gm.dtype).double(), om)
    fo = OH.refine_flags(Uo, om, field, 0.3, 0.075).numpy()
    assert np.array_equal(fg, fo)
    assert (fo == 1).any() and (fo == 0).any()
