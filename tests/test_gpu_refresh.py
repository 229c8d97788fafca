"""GPU ghost refresh (copy, restriction, prolongation, physical boundaries)
against the oracle on AMR meshes."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM

pytestmark = pytest.mark.gpu


def _random_state(om, seed):
    od = om.desc
    U = H.state(od, om.leaves, "blobs", count=20, seed=seed)
    g = torch.Generator().manual_seed(seed)
    U = U * (1.0 + 0.3 * torch.rand(U.shape, generator=g, dtype=torch.float64))
    return U


@pytest.mark.parametrize("seed,bc,n", [
    (0, (OM.PERIODIC,) * 3, 8),
    (1, (OM.OUTFLOW, OM.PERIODIC, OM.OUTFLOW), 16),
    (2, (OM.OUTFLOW,) * 3, 8),
])
def test_refresh_fp64_matches_oracle_bitwise(seed, bc, n):
    od = H.oracle_desc(root=(2, 2, 2), n=n, lmax=2, bc=bc)
    meshes, flags = H.flag_sequence(od, rounds=2, seed=seed, p_refine=0.4)
    om = meshes[-1]
    plan = OH.RefreshPlan(om)
    assert plan.pro_d.numel() > 0 and plan.rst_d.numel() > 0
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    U = _random_state(om, seed)
    Ug = U.cuda().contiguous()
    gm.ghost_refresh(Ug)
    Uo = plan.apply(U)
    assert torch.equal(Ug.cpu(), Uo)


def test_refresh_fp32_close_to_oracle():
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=2, bc=(OM.OUTFLOW, OM.PERIODIC, OM.PERIODIC))
    meshes, flags = H.flag_sequence(od, rounds=2, seed=5, p_refine=0.4)
    om = meshes[-1]
    gm = H.gpu_mesh_from_flags(od, flags, 4)
    U = _random_state(om, 5).float()
    Ug = U.cuda().contiguous()
    gm.ghost_refresh(Ug)
    Uo = OH.ghost_refresh(U.double(), om)
    assert H.rel_err(Ug.cpu(), Uo) < 2e-6


def test_misaligned_state_is_refused_before_any_launch():
    """Every entry point that takes a state pool checks the header's 256-byte
    alignment on the host (the kernels move 16- and 32-byte vectors): a pool
    shifted by one element is refused with CELLO_EINVAL and left untouched."""
    from paper_1810_01319_gb300 import CelloError
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=1)
    gm = H.gpu_mesh_from_flags(od, [np.array([1, 0, 0, 0, 0, 0, 0, 0], dtype=np.int8)], 4)
    raw = torch.zeros(gm.n_leaves * gm.leaf_elems + 1, dtype=torch.float32, device="cuda")
    U = raw[1:].view(gm.n_leaves, gm.nf, gm.N, gm.N, gm.N)
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    for call in (lambda: gm.ghost_refresh(U), lambda: gm.hydro_step(U, dt, 0), lambda: gm.reduce(U, 0.4, dt_next=dt),
                 lambda: gm.refine_flags(U), lambda: gm.reduce_noalloc(U, 0.4, dt_next=dt)):
        with pytest.raises(CelloError):
            call()
    torch.cuda.synchronize()
    assert not raw.any()
