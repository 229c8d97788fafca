"""The multigrid Poisson solver (mg0) on the GPU against the oracle: the same
V-cycles on the same grid give the same potential (max relative difference
1e-12: only the mean removals sum in a different order) and the same
residual history; an odd coarsest grid; unsupported meshes refused."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import mesh as OM
from oracle import poisson as OP

pytestmark = pytest.mark.gpu


def _uniform(root, n, level):
    od = H.oracle_desc(root=(root,) * 3, n=n, lmax=level)
    om = OM.root_mesh(od)
    flags = []
    for _ in range(level):
        f = np.ones(om.n_leaves, dtype=np.int8)
        om = OM.build(od, om, f)
        flags.append(f)
    return od, om, flags


@pytest.mark.parametrize("root,n,level,cycles", [(2, 16, 1, 8), (3, 16, 0, 6)])
def test_poisson_matches_oracle(root, n, level, cycles):
    """float64 cycles: the same arithmetic as the oracle."""
    od, om, flags = _uniform(root, n, level)
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    g = torch.Generator().manual_seed(root * 10 + level)
    f = torch.randn(om.n_leaves, n, n, n, generator=g, dtype=torch.float64)
    phi, res = gm.poisson_solve(f.cuda().contiguous(), cycles)
    M = root * n * (1 << level)
    h = od.dx(level)
    po, ro = OP.solve(OP.to_global(om, f), h, cycles)
    expect = OP.from_global(om, po)
    scale = float(expect.abs().max())
    assert float((phi.cpu() - expect).abs().max()) <= 1e-12 * scale
    assert np.allclose(res, ro, rtol=1e-6, atol=0)
    assert res[-1] < 1e-3 * res[0]
    assert M in (64, 48)


def test_poisson_refuses_amr_and_outflow_meshes():
    from paper_1810_01319_gb300 import CelloError
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=1)
    gm = H.gpu_mesh_from_flags(od, [np.array([1, 0, 0, 0, 0, 0, 0, 0], dtype=np.int8)], 8)
    with pytest.raises(CelloError):
        gm.poisson_solve(torch.zeros(gm.n_leaves, 8, 8, 8, dtype=torch.float64, device="cuda"), 2)
    od2 = H.oracle_desc(root=(2, 2, 2), n=8, lmax=0, bc=(OM.OUTFLOW, OM.PERIODIC, OM.PERIODIC))
    gm2 = H.gpu_mesh_from_flags(od2, [], 8)
    with pytest.raises(CelloError):
        gm2.poisson_solve(torch.zeros(8, 8, 8, 8, dtype=torch.float64, device="cuda"), 2)


@pytest.mark.parametrize("root,n,level", [(2, 16, 1), (3, 16, 0)])
def test_mixed_precision_poisson(root, n, level):
    """float32 cycles on the float64 residual: the residual history follows
    the oracle's mixed-precision cycles (same float32 arithmetic up to the
    mean removal), and 20 cycles reach the float64 discrete solution."""
    od, om, flags = _uniform(root, n, level)
    gm = H.gpu_mesh_from_flags(od, flags, 4)
    g = torch.Generator().manual_seed(root * 7 + level)
    f = torch.randn(om.n_leaves, n, n, n, generator=g, dtype=torch.float64)
    phi, res = gm.poisson_solve(f.cuda().contiguous(), 20, inner=4)
    h = od.dx(level)
    po, ro = OP.solve(OP.to_global(om, f), h, 20, inner="float32")
    p64, _ = OP.solve(OP.to_global(om, f), h, 20)
    expect = OP.from_global(om, p64)
    scale = float(expect.abs().max())
    assert float((phi.cpu() - expect).abs().max()) <= 1e-10 * scale
    assert np.allclose(res[:6], ro[:6], rtol=1e-3, atol=0)
