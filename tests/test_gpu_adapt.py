"""GPU remap and adaptive runs against the oracle (float64, bit-for-bit
meshes, 1e-12 states), and the Sedov-Taylor blast on an adaptive mesh
against the self-similar shock radius."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import exact
from oracle import hydro as OH
from oracle import mesh as OM

pytestmark = pytest.mark.gpu


def test_remap_matches_oracle_bitwise():
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=3, bc=(OM.PERIODIC, OM.OUTFLOW, OM.PERIODIC))
    meshes, flags = H.flag_sequence(od, rounds=2, seed=4, p_refine=0.5)
    old = meshes[-1]
    lv = old.leaves[:, 0]
    rng = np.random.default_rng(0)
    f = np.where(lv == lv.max(), -1, rng.choice([0, 1], size=old.n_leaves, p=[0.6, 0.4])).astype(np.int8)
    new = OM.build(od, old, f)
    g_old = H.gpu_mesh_from_flags(od, flags, 8)
    from paper_1810_01319_gb300 import Mesh
    g_new = Mesh(g_old.desc, g_old, f)
    assert np.array_equal(g_new.leaves.astype(np.int64), new.leaves)
    U = H.state(od, old.leaves, "blobs", count=12, seed=1)
    U = U * (1 + 0.3 * torch.rand(U.shape, generator=torch.Generator().manual_seed(2), dtype=torch.float64))
    Ug = U.cuda().contiguous()
    g_old.ghost_refresh(Ug)
    Vg = g_new.remap_from(g_old, Ug)
    Vo = OH.remap(OH.ghost_refresh(U, old), old, new)
    n, g = od.n, od.ghosts
    assert torch.equal(H.interior(Vg.cpu(), n), H.interior(Vo, n))


def _sedov_initial(od, field=4, tau=0.3):
    mesh = OM.root_mesh(od)
    flags = []
    for _ in range(od.max_level):
        U = OH.ghost_refresh(H.state(od, mesh.leaves, "sedov", max_level=od.max_level), mesh)
        f = OH.refine_flags(U, mesh, field, tau, tau / 4).numpy()
        f = np.where(f > 0, 1, 0).astype(np.int8)
        if not f.any():
            break
        mesh = OM.build(od, mesh, f)
        flags.append(f)
    return mesh, flags


def test_adaptive_sedov_fp64_matches_oracle():
    """Sedov deposit on 2^3 root blocks of 8^3 cells, max level 3, pressure
    slope criterion, adaptation every step: meshes identical and state within
    1e-12 of the oracle over 6 steps."""
    od = OM.Desc(root=(2, 2, 2), n=8, ghosts=4, max_level=3, bc=(OM.PERIODIC,) * 3, gamma=1.4)
    om, flags = _sedov_initial(od)
    U0 = H.state(od, om.leaves, "sedov", max_level=od.max_level)
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    Ug = U0.cuda().contiguous()
    Uo = U0.clone()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    from paper_1810_01319_gb300.drivers import adapt
    for s in range(6):
        om, Uo, _ = OH.adapt(Uo, om, 4, 0.3)
        gm, Ug = adapt(gm, Ug, 4, 0.3)
        assert np.array_equal(gm.leaves.astype(np.int64), om.leaves), s
        d = OH.reduce_dt_totals(Uo, om, 0.4)[0]
        Uo = OH.step(Uo, om, d, s)
        dt.fill_(d)
        gm.hydro_step(Ug, dt, s)
    torch.cuda.synchronize()
    assert om.leaves[:, 0].max() == 3
    err = H.rel_err(H.interior(Ug.cpu(), 8), H.interior(Uo, 8))
    assert err <= 1e-12, err


def _shock_radius(mesh, U, od):
    """Density-weighted mean radius of the cells within 10% of the peak density."""
    from workloads import ics
    x, y, z = ics.cell_centres(mesh.leaves, od.root, od.n, od.ghosts, od.lo, od.hi, device=U.device)
    g, n = od.ghosts, od.n
    sl = (slice(None), slice(g, g + n), slice(g, g + n), slice(g, g + n))
    rho = U[:, 0].double()[sl]
    r = torch.sqrt((x[sl] - 0.5) ** 2 + (y[sl] - 0.5) ** 2 + (z[sl] - 0.5) ** 2)
    m = rho > 0.9 * rho.max()
    return float((r[m] * rho[m]).sum() / rho[m].sum()), float(rho.max())


@pytest.mark.parametrize("precision", [4])
def test_sedov_shock_radius_against_similarity_solution(precision):
    """Sedov-Taylor blast: 2^3 root blocks of 16^3 cells, max level 3,
    pressure-slope refinement every 4 steps, E = 1 in the central 2^3 finest
    cells, rho = 1, p = 1e-5, gamma 1.4, to t = 0.05: the shock radius
    (peak-density shell) is xi0 (E t^2/rho)^(1/5) within 5%, the peak
    density approaches the strong-shock ratio 6."""
    od = OM.Desc(root=(2, 2, 2), n=16, ghosts=4, max_level=3, bc=(OM.PERIODIC,) * 3, gamma=1.4)
    om, flags = _sedov_initial(od)
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    U = H.state(od, om.leaves, "sedov", max_level=od.max_level).to(gm.dtype).cuda().contiguous()
    from paper_1810_01319_gb300.drivers import run_adaptive
    gm, U, t, steps = run_adaptive(gm, U, 0.05, 0.4, field=4, tau=0.3, adapt_every=4)
    assert abs(t - 0.05) < 1e-12
    R, peak = _shock_radius(gm, U, od)
    R_exact = exact.sedov_xi0(1.4) * (0.05 ** 2) ** 0.2
    assert abs(R / R_exact - 1) < 0.05, (R, R_exact, steps)
    assert 3.0 < peak < 6.5
