"""Pins of the oracle's full hydro step (Sec. II.B ghost refresh, Refine /
Restrict / Prolong; Sec. II.C PPM): invariants, conservation, AMR = uniform,
Sod against the exact solution, CFL and totals closed forms, brute-force
refinement flags, prolongation/restriction identities."""
import numpy as np
import pytest
import torch

from oracle import exact
from oracle import hydro as H
from oracle import mesh as M
from workloads import ics


def _sod_mesh(nx_roots, n=16):
    d = M.Desc(root=(nx_roots, 1, 1), n=n, ghosts=4, max_level=0, hi=(1.0, 1.0 / nx_roots, 1.0 / nx_roots),
               bc=(M.OUTFLOW, M.PERIODIC, M.PERIODIC), gamma=1.4)
    return M.root_mesh(d)


def _state(mesh, kind, **kw):
    d = mesh.desc
    f = getattr(ics, kind)
    return f(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi, d.gamma, **kw)


def _interior(mesh, U):
    n, g = mesh.desc.n, mesh.desc.ghosts
    return U[:, :, g:g + n, g:g + n, g:g + n]


def _amr_mesh(root=(2, 2, 2), n=8, lmax=2, seed=0, bc=(M.PERIODIC,) * 3):
    d = M.Desc(root=root, n=n, ghosts=4, max_level=lmax, bc=bc, gamma=5.0 / 3.0,
               hi=tuple(r / max(root) for r in root))
    rng = np.random.default_rng(seed)
    mesh = M.root_mesh(d)
    for _ in range(lmax):
        mesh = M.build(d, mesh, rng.choice([0, 1], size=mesh.n_leaves, p=[0.6, 0.4]))
    return mesh


def test_uniform_state_is_invariant():
    d = M.Desc(root=(2, 2, 2), n=8, ghosts=4, max_level=0, bc=(M.PERIODIC, M.OUTFLOW, M.PERIODIC), gamma=1.4)
    mesh = M.root_mesh(d)
    U = _state(mesh, "uniform", rho=1.3, vel=(0.3, -0.2, 0.1), p=0.7)
    U1, _ = H.run(U, mesh, 3, 0.4)
    assert torch.equal(_interior(mesh, U1), _interior(mesh, U))


def test_uniform_state_on_amr_mesh():
    mesh = _amr_mesh(seed=1)
    assert mesh.leaves[:, 0].max() == 2
    U = _state(mesh, "uniform", rho=1.3, vel=(0.3, -0.2, 0.1), p=0.7)
    U1, _ = H.run(U, mesh, 2, 0.4)
    assert torch.allclose(_interior(mesh, U1), _interior(mesh, U), rtol=1e-14, atol=1e-15)


def test_mirror_symmetry_bit_exact():
    mesh = _sod_mesh(4)
    U = _state(mesh, "sod", x0=0.4)
    # mirror image: reverse the leaf order and the x index, negate x momentum
    Um = U.flip(0).flip(-1).clone()
    Um[:, 1] = -Um[:, 1]
    A, dts = H.run(U, mesh, 10, 0.4)
    Bm, _ = H.run(Um, mesh, 10, 0.4, dts=dts)
    Bb = Bm.flip(0).flip(-1).clone()
    Bb[:, 1] = -Bb[:, 1]
    assert torch.equal(_interior(mesh, A), _interior(mesh, Bb))


def _sod_l1(nx_roots, n=16):
    mesh = _sod_mesh(nx_roots, n)
    U = _state(mesh, "sod")
    U, dts = H.run(U, mesh, 10 * nx_roots, 0.4)
    T = sum(dts)
    g = mesh.desc.ghosts
    rho = torch.cat([_interior(mesh, U)[b, 0, 0, 0, :] for b in range(nx_roots)]).numpy()
    ncell = nx_roots * n
    x = (np.arange(ncell) + 0.5) / ncell
    re, ue, pe = exact.sample((x - 0.5) / T, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    return np.abs(rho - re).mean(), rho, re, x, T


def test_sod_against_exact_solution():
    e64, *_ = _sod_l1(4)
    e128, rho, re, x, T = _sod_l1(8)
    assert e64 < 0.01
    assert e128 < e64 / 2 ** 0.6              # observed order >= 0.6
    # star-region plateau between contact and shock within 1.5%
    ps, us = exact.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    plateau = (x > 0.5 + us * T + 0.025) & (x < 0.5 + 1.75 * T - 0.025)
    assert plateau.sum() >= 3
    assert np.abs(rho[plateau] / re[plateau] - 1).max() < 0.015


def test_transverse_invariance_of_sod():
    mesh = _sod_mesh(2)
    U, _ = H.run(_state(mesh, "sod"), mesh, 5, 0.4)
    I = _interior(mesh, U)
    assert torch.equal(I, I[:, :, :1, :1, :].expand_as(I))


def test_all_one_level_amr_equals_uniform_grid():
    g = 4
    # uniform grid: one 32^3 block;  AMR: one root refined once into 8 leaves of 16^3
    dA = M.Desc(root=(1, 1, 1), n=32, ghosts=g, max_level=0, gamma=5.0 / 3.0)
    dB = M.Desc(root=(1, 1, 1), n=16, ghosts=g, max_level=1, gamma=5.0 / 3.0)
    mA = M.root_mesh(dA)
    mB = M.build(dB, M.root_mesh(dB), [1])
    assert mB.n_leaves == 8
    UA = ics.blobs(mA.leaves, dA.root, dA.n, g, dA.lo, dA.hi, dA.gamma, count=6, seed=3)
    UB = ics.blobs(mB.leaves, dB.root, dB.n, g, dB.lo, dB.hi, dB.gamma, count=6, seed=3)
    A, dts = H.run(UA, mA, 3, 0.4)
    B, _ = H.run(UB, mB, 3, 0.4, dts=dts)
    IA = A[0, :, g:g + 32, g:g + 32, g:g + 32]
    for b, (L, i, j, k) in enumerate(mB.leaves):
        sl = IA[:, 16 * k:16 * k + 16, 16 * j:16 * j + 16, 16 * i:16 * i + 16]
        assert torch.equal(B[b, :, g:g + 16, g:g + 16, g:g + 16], sl)


def _totals(mesh, U):
    return H.reduce_dt_totals(U, mesh, 0.4)[1]


def test_conservation_on_periodic_amr_mesh():
    mesh = _amr_mesh(seed=2)
    d = mesh.desc
    assert len(H.coarse_fine_faces(mesh)) > 0
    U = ics.blobs(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi, d.gamma, count=12, seed=5)
    T0 = _totals(mesh, U)
    U1, dts = H.run(U, mesh, 3, 0.4)
    T1 = _totals(mesh, U1)
    scale = _totals(mesh, U.abs())
    assert ((T1 - T0).abs() / scale).max() < 1e-13
    # negative control: without the coarse-fine flux correction mass drifts
    plan = H.RefreshPlan(mesh)
    V = U
    for s, dt in enumerate(dts):
        V = H.step(V, mesh, dt, s, plan, flux_correction=False)
    assert ((_totals(mesh, V) - T0).abs() / scale)[0] > 1e-9


def test_dt_closed_form():
    d = M.Desc(root=(2, 1, 1), n=8, ghosts=4, max_level=0, hi=(1.0, 0.5, 0.5), gamma=1.4)
    mesh = M.root_mesh(d)
    U = _state(mesh, "uniform", rho=2.0, vel=(0.1, -0.7, 0.3), p=3.0)
    dt, tot = H.reduce_dt_totals(U, mesh, 0.4)
    c = np.sqrt(1.4 * 3.0 / 2.0)
    assert dt == pytest.approx(0.4 * (1.0 / 16) / (0.7 + c), rel=1e-14)
    vol = 0.25
    E = 3.0 / 0.4 + 0.5 * 2.0 * (0.01 + 0.49 + 0.09)
    assert tot.numpy() == pytest.approx(np.array([2.0, 0.2, -1.4, 0.6, E]) * vol, rel=1e-13)


def test_totals_closed_form_sod():
    mesh = _sod_mesh(4)
    tot = _totals(mesh, _state(mesh, "sod"))
    area = 0.25 * 0.25
    assert float(tot[0]) == pytest.approx(area * (0.5 * 1.0 + 0.5 * 0.125), rel=1e-14)
    assert float(tot[4]) == pytest.approx(area * (0.5 * 2.5 + 0.5 * 0.25), rel=1e-14)


def test_refine_flags_brute_force():
    mesh = _amr_mesh(root=(2, 1, 1), n=8, lmax=2, seed=4)
    d = mesh.desc
    U = ics.blobs(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi, d.gamma, count=10, seed=7)
    U = H.ghost_refresh(U, mesh)
    for field in (0, 4):
        flags = H.refine_flags(U, mesh, field, 0.3, 0.075)
        n, g = d.n, d.ghosts
        for b in range(mesh.n_leaves):
            L = int(mesh.leaves[b, 0])
            Ub = U[b].numpy()
            if field == 0:
                q = np.maximum(Ub[0], 1e-10)
            else:
                rho = np.maximum(Ub[0], 1e-10)
                u, v, w = Ub[1] / rho, Ub[2] / rho, Ub[3] / rho
                q = np.maximum((d.gamma - 1) * (Ub[4] - 0.5 * rho * (u * u + (v * v + w * w))), 1e-20)
            hit = hit_c = False
            for z in range(g, g + n):
                for y in range(g, g + n):
                    for x in range(g, g + n):
                        for (a, b2) in (((z, y, x + 1), (z, y, x - 1)), ((z, y + 1, x), (z, y - 1, x)),
                                        ((z + 1, y, x), (z - 1, y, x))):
                            diff = abs(q[a] - q[b2])
                            hit |= diff > 0.6 * abs(q[z, y, x])
                            hit_c |= diff > 0.15 * abs(q[z, y, x])
            want = 1 if (hit and L < d.max_level) else (-1 if (not hit_c and L > 0) else 0)
            assert int(flags[b]) == want


def test_refresh_reproduces_linear_fields():
    """Copy, restriction and limited prolongation are all exact on a linear
    field (minmod of equal differences is that difference)."""
    mesh = _amr_mesh(root=(1, 1, 1), n=8, lmax=2, seed=7, bc=(M.OUTFLOW,) * 3)
    d = mesh.desc
    x, y, z = ics.cell_centres(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)
    lin = 1.0 + 0.5 * x - 0.25 * y + 0.125 * z
    U = torch.stack([lin, 2 * lin, -lin, 0.5 * lin, 3 * lin], 1).contiguous()
    n, g = d.n, d.ghosts
    garbage = U.clone()
    inner = torch.zeros_like(U, dtype=torch.bool)
    inner[:, :, g:g + n, g:g + n, g:g + n] = True
    garbage[~inner] = 123.0
    plan = H.RefreshPlan(mesh)
    assert plan.copy_d.numel() and plan.rst_d.numel() and plan.pro_d.numel()
    R = plan.apply(garbage)
    ok = (x > 0.2) & (x < 0.8) & (y > 0.2) & (y < 0.8) & (z > 0.2) & (z < 0.8)
    ok = ok.unsqueeze(1).expand_as(U)
    assert (R[ok] - U[ok]).abs().max() < 1e-14
    assert (R != 123.0).all()


def test_prolong_restrict_identities():
    """Restriction of the eight prolonged children returns the parent, and
    their mean equals it (conservation), up to round-off."""
    g = torch.Generator().manual_seed(3)
    Uc, Um, Up = torch.rand(3, 3, 1000, generator=g, dtype=torch.float64)
    D = [H.minmod(Uc[a] - Um[a], Up[a] - Uc[a]) for a in range(3)]
    kids = []
    for dz in (-1.0, 1.0):
        for dy in (-1.0, 1.0):
            for dx in (-1.0, 1.0):
                kids.append(Uc[0] + 0.25 * ((dx * D[0] + dy * D[1]) + dz * D[2]))
    s = kids[0]
    for k in kids[1:]:
        s = s + k
    assert ((s * 0.125) - Uc[0]).abs().max() < 1e-15


def test_remap_conserves_and_reproduces_linear_fields():
    d = M.Desc(root=(2, 2, 2), n=8, ghosts=4, max_level=3, bc=(M.PERIODIC,) * 3, gamma=1.4)
    rng = np.random.default_rng(3)
    old = M.root_mesh(d)
    for _ in range(2):
        old = M.build(d, old, rng.choice([0, 1], size=old.n_leaves, p=[0.5, 0.5]))
    lv = old.leaves[:, 0]
    flags = np.where(lv == lv.max(), -1, rng.choice([0, 1], size=old.n_leaves, p=[0.6, 0.4])).astype(np.int8)
    new = M.build(d, old, flags)
    kinds = set()
    for t in map(tuple, new.leaves.tolist()):
        kinds.add("copy" if t in old.index else ("restrict" if all(
            (t[0] + 1, 2 * t[1] + (o & 1), 2 * t[2] + ((o >> 1) & 1), 2 * t[3] + (o >> 2)) in old.index
            for o in range(8)) else "prolong"))
    assert kinds == {"copy", "restrict", "prolong"}
    U = ics.blobs(old.leaves, d.root, d.n, d.ghosts, d.lo, d.hi, d.gamma, count=8, seed=2)
    U = H.ghost_refresh(U, old)
    V = H.remap(U, old, new)
    scale = _totals(old, U.abs())
    assert ((_totals(new, V) - _totals(old, U)).abs() / scale).max() < 1e-14
    # a linear field (away from the periodic seam) is reproduced exactly
    x, y, z = ics.cell_centres(old.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)
    lin = lambda x, y, z: 1.0 + 0.5 * x - 0.25 * y + 0.125 * z
    Ul = torch.stack([lin(x, y, z)] * 5, 1).contiguous()
    Ul = H.ghost_refresh(Ul, old)
    Vl = H.remap(Ul, old, new)
    xn, yn, zn = ics.cell_centres(new.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)
    g, n = d.ghosts, d.n
    want = lin(xn, yn, zn)[:, g:g + n, g:g + n, g:g + n]
    got = Vl[:, 0, g:g + n, g:g + n, g:g + n]
    inner = ((xn > 0.2) & (xn < 0.8) & (yn > 0.2) & (yn < 0.8) & (zn > 0.2) & (zn < 0.8))[:, g:g + n, g:g + n, g:g + n]
    assert inner.sum() > 1000
    assert (got - want)[inner].abs().max() < 1e-14


def test_sod_with_hllc_against_exact_solution():
    """The HLLC interface flux in the full PPM step: Sod converges to the
    exact solution like the two-shock flux does."""
    errs = []
    for nx in (4, 8):
        d = M.Desc(root=(nx, 1, 1), n=16, ghosts=4, max_level=0, hi=(1.0, 1.0 / nx, 1.0 / nx),
                   bc=(M.OUTFLOW, M.PERIODIC, M.PERIODIC), gamma=1.4, riemann="hllc")
        mesh = M.root_mesh(d)
        U, dts = H.run(_state(mesh, "sod"), mesh, 10 * nx, 0.4)
        T = sum(dts)
        rho = torch.cat([_interior(mesh, U)[b, 0, 0, 0, :] for b in range(nx)]).numpy()
        x = (np.arange(nx * 16) + 0.5) / (nx * 16)
        re, _, _ = exact.sample((x - 0.5) / T, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
        errs.append(np.abs(rho - re).mean())
    assert errs[0] < 0.01 and errs[1] < errs[0] / 2 ** 0.6, errs


def _contact_run(steepen, steps=40):
    """A density step (contact: uniform p = 1, u = 0.5) advected across a
    periodic x box of 4 x 16 cells."""
    d = M.Desc(root=(4, 1, 1), n=16, ghosts=4, max_level=0, hi=(1.0, 0.25, 0.25), gamma=1.4, steepen=steepen)
    mesh = M.root_mesh(d)
    x, _, _ = ics.cell_centres(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)
    rho = torch.where((x > 0.25) & (x < 0.5), torch.full_like(x, 1.0), torch.full_like(x, 0.125))
    U = ics.conserved(rho, 0.5 * torch.ones_like(x), 0 * x, 0 * x, torch.ones_like(x), 1.4)
    dts = [0.004] * steps
    U1, _ = H.run(U, mesh, steps, 0.4, dts=dts)
    r = torch.cat([_interior(mesh, U1)[b, 0, 0, 0, :] for b in range(4)])
    xc = (torch.arange(64, dtype=torch.float64) + 0.5) / 64
    shift = 0.5 * 0.004 * steps
    exact = torch.where(((xc - shift) % 1.0 > 0.25) & ((xc - shift) % 1.0 < 0.5), 1.0, 0.125)
    return r, exact


def test_contact_steepening_sharpens_an_advected_contact():
    r0, exact = _contact_run(False)
    r1, _ = _contact_run(True)
    mid0 = int(((r0 > 0.2) & (r0 < 0.9)).sum())
    mid1 = int(((r1 > 0.2) & (r1 < 0.9)).sum())
    assert mid1 < mid0, (mid0, mid1)
    assert float((r1 - exact).abs().mean()) < float((r0 - exact).abs().mean())
    # mass is conserved either way (periodic box)
    assert abs(float(r1.sum()) - float(r0.sum())) < 1e-12 * float(r0.sum())


def test_steepening_keeps_uniform_states_and_mirror_symmetry():
    d = M.Desc(root=(2, 2, 2), n=8, ghosts=4, max_level=0, bc=(M.PERIODIC, M.OUTFLOW, M.PERIODIC), gamma=1.4,
               steepen=True)
    mesh = M.root_mesh(d)
    U = _state(mesh, "uniform", rho=1.3, vel=(0.3, -0.2, 0.1), p=0.7)
    U1, _ = H.run(U, mesh, 3, 0.4)
    assert torch.equal(_interior(mesh, U1), _interior(mesh, U))
    d2 = M.Desc(root=(4, 1, 1), n=16, ghosts=4, max_level=0, hi=(1.0, 0.25, 0.25),
                bc=(M.OUTFLOW, M.PERIODIC, M.PERIODIC), gamma=1.4, steepen=True)
    mesh = M.root_mesh(d2)
    U = _state(mesh, "sod", x0=0.4)
    Um = U.flip(0).flip(-1).clone()
    Um[:, 1] = -Um[:, 1]
    A, dts = H.run(U, mesh, 10, 0.4)
    Bm, _ = H.run(Um, mesh, 10, 0.4, dts=dts)
    Bb = Bm.flip(0).flip(-1).clone()
    Bb[:, 1] = -Bb[:, 1]
    assert torch.equal(_interior(mesh, A), _interior(mesh, Bb))


def test_refresh_plan_on_a_subset_of_leaves():
    """A plan restricted to some destination leaves, compacted onto a pool of
    just the leaves it reads, fills those leaves' ghosts exactly as the
    full plan does (the sampled full-size GPU parity test relies on it)."""
    d = M.Desc(root=(2, 2, 2), n=8, ghosts=4, max_level=2, gamma=5.0 / 3.0, hi=(1.0, 1.0, 1.0),
               bc=(M.PERIODIC, M.OUTFLOW, M.PERIODIC))
    rng = np.random.default_rng(4)
    mesh = M.root_mesh(d)
    for _ in range(2):
        mesh = M.build(d, mesh, rng.choice([0, 1], size=mesh.n_leaves, p=[0.6, 0.4]).astype(np.int8))
    U = _state(mesh, "blobs", count=6, seed=1)
    full = H.ghost_refresh(U, mesh)
    dest = sorted(set(int(b) for b in rng.choice(mesh.n_leaves, 6, replace=False)))
    plan = H.RefreshPlan(mesh, dest=dest)
    read = plan.leaves_read()
    assert set(dest) <= set(read.tolist()) and len(read) < mesh.n_leaves
    out = plan.compact(read).apply(U[torch.as_tensor(read)].clone())
    for k, b in enumerate(read):
        if b in dest:
            assert torch.equal(out[k], full[b])
