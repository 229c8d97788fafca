"""Pins of the oracle's tracer particles (Sec. II.B: particles move between
Blocks; Sec. III: tracers in the hydro workload): leaf lookup against brute
force, trilinear interpolation exact on linear fields across levels,
uniform-flow advection with periodic wrap and migration, outflow loss."""
import numpy as np
import torch

from oracle import mesh as M
from oracle import particles as P
from workloads import ics


def _amr(bc=(M.PERIODIC,) * 3, seed=0):
    d = M.Desc(root=(2, 2, 2), n=8, ghosts=4, max_level=2, bc=bc, gamma=1.4)
    rng = np.random.default_rng(seed)
    mesh = M.root_mesh(d)
    for _ in range(2):
        mesh = M.build(d, mesh, rng.choice([0, 1], size=mesh.n_leaves, p=[0.6, 0.4]))
    assert mesh.leaves[:, 0].max() == 2 and mesh.leaves[:, 0].min() < 2
    return d, mesh


def _points(n, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.rand(3, n, generator=g, dtype=torch.float64)


def test_locate_matches_brute_force_containment():
    d, mesh = _amr()
    pos = _points(400, 1)
    leaf = P.locate(mesh, pos)
    for p in range(pos.shape[1]):
        hits = []
        for b, (L, i, j, k) in enumerate(mesh.leaves):
            w = (d.hi[0] - d.lo[0]) / d.root[0] / (1 << int(L))
            lo = [d.lo[a] + idx * w for a, idx in enumerate((i, j, k))]
            if all(lo[a] <= float(pos[a, p]) < lo[a] + w for a in range(3)):
                hits.append(b)
        assert hits == [int(leaf[p])]


def _linear_state(mesh, A, c):
    """rho = 1 + 0.1 x, momentum = rho * (A x + c), sampled at every cell
    centre (ghosts included), so the velocity is exactly linear."""
    d = mesh.desc
    x, y, z = ics.cell_centres(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)
    X = torch.stack([x, y, z])
    rho = 1.0 + 0.1 * x
    vel = [c[a] + A[a][0] * x + A[a][1] * y + A[a][2] * z for a in range(3)]
    return ics.conserved(rho, vel[0], vel[1], vel[2], torch.ones_like(x), d.gamma), X


def test_trilinear_velocity_is_exact_on_linear_fields():
    d, mesh = _amr(seed=2)
    A = [[0.3, -0.2, 0.1], [0.05, 0.4, -0.3], [-0.1, 0.2, 0.25]]
    c = [0.1, -0.2, 0.3]
    U, _ = _linear_state(mesh, A, c)
    pos = 0.05 + 0.9 * _points(300, 3)
    leaf = P.locate(mesh, pos)
    vel = P.velocity(U, mesh, pos, leaf)
    for a in range(3):
        exact = c[a] + A[a][0] * pos[0] + A[a][1] * pos[1] + A[a][2] * pos[2]
        assert float((vel[a] - exact).abs().max()) < 1e-13


def test_uniform_flow_translates_wraps_and_migrates():
    d, mesh = _amr(seed=3)
    x, _, _ = ics.cell_centres(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)
    one = torch.ones_like(x)
    u = (0.31, -0.17, 0.23)
    U = ics.conserved(one, u[0] * one, u[1] * one, u[2] * one, one, d.gamma)
    pos = _points(500, 4)
    leaf = P.locate(mesh, pos)
    dt = 0.05
    p1, l1 = P.push(U, mesh, pos, leaf, dt)
    assert bool((l1 >= 0).all())
    for a in range(3):
        moved = pos[a] + dt * u[a]
        wrapped = torch.where(moved < 0.0, moved + 1.0, torch.where(moved >= 1.0, moved - 1.0, moved))
        assert torch.allclose(p1[a], wrapped, rtol=0, atol=1e-15)
    assert torch.equal(l1, P.locate(mesh, p1))
    assert int((l1 != leaf).sum()) > 50          # many tracers crossed a Block face
    # back again with the opposite flow
    Ub = ics.conserved(one, -u[0] * one, -u[1] * one, -u[2] * one, one, d.gamma)
    p2, l2 = P.push(Ub, mesh, p1, l1, dt)
    assert float((p2 - pos).abs().max()) < 1e-14
    assert torch.equal(l2, leaf) or int((l2 != leaf).sum()) <= 2   # points within rounding of a face


def test_outflow_loses_tracers_that_leave():
    d, mesh = _amr(bc=(M.OUTFLOW, M.PERIODIC, M.PERIODIC), seed=4)
    x, _, _ = ics.cell_centres(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)
    one = torch.ones_like(x)
    U = ics.conserved(one, 0.5 * one, 0 * one, 0 * one, one, d.gamma)
    pos = _points(300, 5)
    leaf = P.locate(mesh, pos)
    p1, l1 = P.push(U, mesh, pos, leaf, 0.1)
    lost = pos[0] + 0.1 * 0.5 >= 1.0
    assert torch.equal(l1 < 0, lost)
    p2, l2 = P.push(U, mesh, p1, l1, 0.1)
    assert torch.equal(p2[:, lost], p1[:, lost])   # lost tracers stay put
