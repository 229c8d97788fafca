"""Pins of the oracle's dual-energy formalism (the modified PPM of Sec. II.C
cites Bryan et al. 1995, whose dual-energy formalism carries the internal
energy density rho e as a sixth field): the pressure selection in closed
form, identity with the plain method on hot flows, invariance of a cold
uniform flow, entropy kept in a cold isentropic compression where the plain
method loses it, conservation on periodic AMR meshes, and a refresh and remap
that treat the sixth field like the others."""
import math

import numpy as np
import pytest
import torch

from oracle import hydro as H
from oracle import mesh as M
from workloads import ics


def _desc(root=(2, 2, 2), n=8, lmax=2, dual=True, riemann="two-shock", bc=(M.PERIODIC,) * 3, hi=None):
    return M.Desc(root=root, n=n, ghosts=4, max_level=lmax, bc=bc, gamma=5.0 / 3.0,
                  hi=hi or tuple(r / max(root) for r in root), riemann=riemann, dual_energy=dual)


def _amr(desc, seed):
    rng = np.random.default_rng(seed)
    mesh = M.root_mesh(desc)
    for _ in range(desc.max_level):
        mesh = M.build(desc, mesh, rng.choice([0, 1], size=mesh.n_leaves, p=[0.6, 0.4]))
    return mesh


def _interior(mesh, U):
    n, g = mesh.desc.n, mesh.desc.ghosts
    return U[:, :, g:g + n, g:g + n, g:g + n]


def test_pressure_selection_closed_form():
    """p = (gamma - 1)(E - ke) where E - ke > DE_ETA1 E, else (gamma - 1) rho e;
    e = rho e / rho."""
    g = 1.4
    f64 = dict(dtype=torch.float64)
    rho = torch.tensor([2.0, 2.0], **f64)
    u = torch.tensor([3.0, 3.0], **f64)
    ke = 0.5 * 2.0 * 9.0
    E = torch.tensor([ke / (1 - 2e-3), ke / (1 - 0.5e-3)], **f64)   # E - ke = 2e-3 E and 0.5e-3 E
    rhoe = torch.tensor([7e-3, 7e-3], **f64)
    z = torch.zeros(2, **f64)
    W = H.primitives(rho, rho * u, z, z, E, g, rhoe=rhoe)
    assert len(W) == 6
    assert math.isclose(float(W[4][0]), (g - 1.0) * (float(E[0]) - ke), rel_tol=1e-12)
    assert float(W[4][1]) == (g - 1.0) * 7e-3
    assert float(W[5][0]) == 7e-3 / 2.0
    # without rho e: the plain formula
    assert math.isclose(float(H.primitives(rho, rho * u, z, z, E, g)[4][1]), (g - 1.0) * (float(E[1]) - ke),
                        rel_tol=1e-9)


@pytest.mark.parametrize("riemann", ["two-shock", "hllc"])
def test_hot_flow_matches_plain_method(riemann):
    """Where E - ke exceeds DE_ETA1 E in every cell the pressure never comes
    from rho e, so the five conserved fields are bit-identical to the plain
    method's; where it exceeds DE_ETA2 E after every sweep, rho e ends equal
    to E - ke, except in the coarse cells beside a finer leaf, where the flux
    correction that follows the sweeps corrects rho e and E each by its own
    fluxes."""
    d6 = _desc(riemann=riemann)
    mesh6 = _amr(d6, 3)
    mesh5 = _amr(_desc(riemann=riemann, dual=False), 3)       # the same flags: the same leaves
    assert np.array_equal(mesh5.leaves, mesh6.leaves)
    U5 = ics.blobs(mesh6.leaves, d6.root, d6.n, d6.ghosts, d6.lo, d6.hi, d6.gamma, count=12, seed=5)
    U6 = ics.with_internal_energy(U5)
    eint = U6[:, 5]
    assert float((eint / U6[:, 4]).min()) > 0.3
    A, dts = H.run(U5, mesh5, 3, 0.4)
    B, _ = H.run(U6, mesh6, 3, 0.4, dts=dts)
    assert torch.equal(_interior(mesh6, B)[:, :5], _interior(mesh5, A))
    I = _interior(mesh6, B)
    ke = 0.5 * (I[:, 1] ** 2 + I[:, 2] ** 2 + I[:, 3] ** 2) / I[:, 0]
    off = ((I[:, 5] - (I[:, 4] - ke)).abs() / I[:, 4]) > 1e-13
    corrected = torch.zeros_like(off)
    n = d6.n
    for b, axis, side, _ in H.coarse_fine_faces(mesh6):
        idx = [b, slice(None), slice(None), slice(None)]
        idx[3 - axis] = n - 1 if side > 0 else 0
        corrected[tuple(idx)] = True
    assert corrected.any() and off.any()
    assert not (off & ~corrected).any()


def test_cold_uniform_flow_is_invariant():
    """A uniform flow at Mach ~ 3000 (pressure from rho e) stays uniform,
    rho e included, on an AMR mesh."""
    d = _desc()
    mesh = _amr(d, 1)
    U = ics.with_internal_energy(ics.uniform(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi, d.gamma,
                                             rho=1.3, vel=(3.0, -2.0, 1.0), p=1e-6))
    I0 = _interior(mesh, U)
    assert float((I0[:, 5] / I0[:, 4]).max()) < 1e-3        # the rho e branch
    U1, _ = H.run(U, mesh, 2, 0.4)
    assert torch.allclose(_interior(mesh, U1), I0, rtol=1e-13, atol=1e-18)


def _compression(dual, steps=30):
    """1-D periodic cold flow u = 1 + 0.5 sin(2 pi x), rho = 1, p = 1e-6
    (Mach ~ 1000, kinetic energy above DE_ETA2 of the total everywhere, so
    rho e is never reset): smooth compression and expansion, no shock before
    t ~ 1/pi.  Returns (max |K / K0 - 1| of the entropy K = p / rho^gamma,
    max |rho - 1|) after the steps."""
    d = _desc(root=(8, 1, 1), n=16, lmax=0, dual=dual, hi=(1.0, 0.125, 0.125))
    mesh = M.root_mesh(d)
    x = ics.cell_centres(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)[0]
    one = torch.ones_like(x)
    p0 = 1e-6
    U = ics.conserved(one, 1.0 + 0.5 * torch.sin(2 * math.pi * x), 0 * x, 0 * x, p0 * one, d.gamma)
    if dual:
        U = ics.with_internal_energy(U)
    U1, _ = H.run(U, mesh, steps, 0.4)
    I = _interior(mesh, U1)
    p = H.lab_primitives(I, d.gamma)[4]
    K = p / I[:, 0] ** d.gamma
    return float((K / p0 - 1.0).abs().max()), float((I[:, 0] - 1).abs().max())


def test_isentropic_compression_keeps_entropy():
    """The compression term -p div(u) of the internal-energy equation keeps
    the entropy of a smooth cold flow (to truncation error, here below 1 %)
    while density changes by a quarter; with the sign of that term reversed
    the error is about 0.3, and the plain method, whose pressure is the
    small difference E - ke, misses the entropy by a factor of about 100."""
    err_de, drho = _compression(True)
    err_plain, _ = _compression(False)
    assert drho > 0.2
    assert err_de < 0.01
    assert err_plain > 100 * err_de


def test_conservation_with_dual_energy():
    """The five conserved totals on a periodic AMR mesh are kept to rounding
    with dual energy on; the blob field is cold enough that both pressure
    branches are taken."""
    d = _desc()
    mesh = _amr(d, 2)
    assert len(H.coarse_fine_faces(mesh)) > 0
    U = ics.with_internal_energy(ics.blobs(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi, d.gamma,
                                           count=12, seed=5, p0=1e-4))
    I = _interior(mesh, U)
    frac = I[:, 5] / I[:, 4]
    assert float(frac.min()) < H.DE_ETA1 and float(frac.max()) > H.DE_ETA2
    T0 = H.reduce_dt_totals(U, mesh, 0.4)[1]
    assert T0.shape == (5,)
    U1, _ = H.run(U, mesh, 3, 0.4)
    T1 = H.reduce_dt_totals(U1, mesh, 0.4)[1]
    scale = H.reduce_dt_totals(U.abs(), mesh, 0.4)[1]
    assert ((T1 - T0).abs() / scale).max() < 1e-13


def test_refresh_and_remap_treat_the_sixth_field_like_the_others():
    """Ghost refresh and remap act field by field: the sixth field of a
    dual-energy state comes out as field 0 of a plain state carrying the
    same values."""
    d6 = _desc()
    mesh6 = _amr(d6, 4)
    mesh5 = _amr(_desc(dual=False), 4)
    assert np.array_equal(mesh5.leaves, mesh6.leaves)
    U5 = ics.blobs(mesh6.leaves, d6.root, d6.n, d6.ghosts, d6.lo, d6.hi, d6.gamma, count=12, seed=6)
    g = torch.Generator().manual_seed(3)
    extra = torch.rand(U5[:, :1].shape, generator=g, dtype=torch.float64) + 0.5
    U6 = torch.cat([U5, extra], 1)
    V5 = U5.clone()
    V5[:, 0] = extra[:, 0]
    R6 = H.ghost_refresh(U6, mesh6)
    R5 = H.ghost_refresh(V5, mesh5)
    assert torch.equal(R6[:, 5], R5[:, 0])
    assert torch.equal(R6[:, 1:5], R5[:, 1:5])
    flags = np.random.default_rng(7).choice([-1, 0, 1], size=mesh6.n_leaves).astype(np.int8)
    new6 = M.build(d6, mesh6, flags)
    new5 = M.build(mesh5.desc, mesh5, flags)
    assert np.array_equal(new6.leaves, new5.leaves) and not np.array_equal(new6.leaves, mesh6.leaves)
    A6 = H.remap(R6, mesh6, new6)
    A5 = H.remap(R5, mesh5, new5)
    assert A6.shape[1] == 6
    assert torch.equal(A6[:, 5], A5[:, 0])


@pytest.mark.parametrize("riemann", ["two-shock", "hllc"])
def test_cold_contact_keeps_pressure_near_uniform(riemann):
    """A density step (1 to 0.25) advected at Mach ~ 1000 with uniform
    pressure: rho e takes the mass flux times the e of the upwind state, so
    the pressure from rho e stays within 20 % of uniform (the separate
    reconstructions of rho and e leave a few per cent at the contact).
    Taking e from the downwind state drives it to ~3e4."""
    d = _desc(root=(8, 1, 1), n=16, lmax=0, hi=(1.0, 0.125, 0.125), riemann=riemann)
    mesh = M.root_mesh(d)
    x = ics.cell_centres(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi)[0]
    one = torch.ones_like(x)
    p0 = 1e-6
    rho = torch.where((x > 0.25) & (x < 0.5), 0.25 * one, one)
    U = ics.with_internal_energy(ics.conserved(rho, one, 0 * x, 0 * x, p0 * one, d.gamma))
    U1, _ = H.run(U, mesh, 20, 0.4)
    I = _interior(mesh, U1)
    p = H.lab_primitives(I, d.gamma)[4]
    assert float((p / p0 - 1).abs().max()) < 0.2
    assert float((I[:, 5] / I[:, 4]).max()) < H.DE_ETA1          # pressure from rho e throughout


def _pencils(seed, B=6, N=24):
    """Random hot pencils (rho, m_n, m_t1, m_t2, E) of length N with jumps."""
    g = torch.Generator().manual_seed(seed)
    r = lambda lo, hi: lo + (hi - lo) * torch.rand(B, 1, N, generator=g, dtype=torch.float64)
    rho, u, v, w, p = r(0.2, 2.0), r(-1.5, 1.5), r(-1.0, 1.0), r(-1.0, 1.0), r(0.2, 2.0)
    return list(ics.conserved(rho, u, v, w, p, 5.0 / 3.0).unbind(1))


@pytest.mark.parametrize("riemann", ["two-shock", "hllc"])
def test_sixth_field_rides_like_a_transverse_velocity(riemann):
    """With rho e set to rho u_t1 (so e = u_t1 exactly) on hot pencils (the
    pressure always from E), the flux of rho e equals the flux of m_t1 bit
    for bit: e is reconstructed, flattened, traced along the entropy wave and
    passed through either solver exactly like a transverse velocity.  The
    other five fluxes are those of the plain method."""
    Uc = _pencils(11)
    dtdx = torch.full((6, 1, 1), 0.3, dtype=torch.float64)
    F5 = H.pencil_fluxes(Uc, dtdx, 5.0 / 3.0, riemann)
    F, u, p = H.pencil_fluxes(Uc + [Uc[2].clone()], dtdx, 5.0 / 3.0, riemann, dual=True)
    assert len(F) == 6
    assert torch.equal(F[5], F[2])
    for k in range(5):
        assert torch.equal(F[k], F5[k])
    assert torch.equal(p, H.primitives(*Uc, 5.0 / 3.0)[4])


def test_hllc_interface_velocity_identity():
    """HLLC: the mass flux is the density of the sampled region's state times
    the interface velocity returned with it (u_K outside the fan, S* inside
    it: rho*_K S* = F*_K of the density by Toro eq. 10.38), and the rho e flux
    is the mass flux times the e of the side the contact leaves behind."""
    g = torch.Generator().manual_seed(5)
    r = lambda lo, hi: lo + (hi - lo) * torch.rand(4000, generator=g, dtype=torch.float64)
    WL = [r(0.2, 2.0), r(-2.0, 2.0), r(-1, 1), r(-1, 1), r(0.1, 2.0), r(0.5, 3.0)]
    WR = [r(0.2, 2.0), r(-2.0, 2.0), r(-1, 1), r(-1, 1), r(0.1, 2.0), r(0.5, 3.0)]
    F, u = H.hllc_flux(WL, WR, 1.4, velocity=True)
    h = H.hllc_waves(WL, WR, 1.4)
    SL, Ss, SR = h["SL"], h["Ss"], h["SR"]
    rho = torch.where(SL >= 0.0, WL[0], torch.where(Ss >= 0.0, h["UsL"][0], torch.where(SR > 0.0, h["UsR"][0], WR[0])))
    assert torch.allclose(rho * u, F[0], rtol=1e-12, atol=1e-12)
    e = torch.where(Ss >= 0.0, WL[5], WR[5])
    assert torch.allclose(F[0] * e, F[5], rtol=1e-12, atol=1e-12)
    star = (SL < 0.0) & (SR > 0.0)
    assert int(star.sum()) > 1000 and int((~star).sum()) > 100


@pytest.mark.parametrize("frac,reset", [(0.2, True), (0.05, False), (5e-4, False)])
def test_sync_rule_closed_form(frac, reset):
    """A uniform flow whose rho e is half its E - ke: the sweeps leave every
    field unchanged (equal fluxes, no velocity difference), then the
    synchronisation sets rho e to E - ke where (E - ke) / E > DE_ETA2 and
    keeps it elsewhere."""
    d = _desc(lmax=0)
    mesh = M.root_mesh(d)
    ke = 0.5 * 1.0 * (1.0 + 0.25 + 0.0625)
    p = (d.gamma - 1.0) * ke * frac / (1.0 - frac)
    U = ics.with_internal_energy(ics.uniform(mesh.leaves, d.root, d.n, d.ghosts, d.lo, d.hi, d.gamma,
                                             rho=1.0, vel=(1.0, 0.5, 0.25), p=p))
    eint = U[:, 5].clone()
    U[:, 5] = 0.5 * eint
    U1 = H.step(U, mesh, 1e-3, 0)
    I0, I1 = _interior(mesh, U), _interior(mesh, U1)
    assert torch.equal(I1[:, :5], I0[:, :5])
    e1 = I1[:, 5]
    if reset:
        assert torch.allclose(e1, _interior(mesh, eint.unsqueeze(1))[:, 0], rtol=1e-12, atol=0)
    else:
        assert torch.equal(e1, I0[:, 5])


def test_two_shock_interface_velocity_identity():
    """Two-shock: the fluxes are the physical fluxes of one state moving at
    the returned interface velocity u (the sampled state): with r = F_rho / u,
    p = F_m - F_rho u, t_k = F_tk / F_rho, the energy flux is u (E + p),
    E = p / (gamma - 1) + r (u^2 + t1^2 + t2^2) / 2."""
    g = torch.Generator().manual_seed(6)
    r_ = lambda lo, hi: lo + (hi - lo) * torch.rand(4000, generator=g, dtype=torch.float64)
    WL = [r_(0.2, 2.0), r_(-2.0, 2.0), r_(-1, 1), r_(-1, 1), r_(0.1, 2.0), r_(0.5, 3.0)]
    WR = [r_(0.2, 2.0), r_(-2.0, 2.0), r_(-1, 1), r_(-1, 1), r_(0.1, 2.0), r_(0.5, 3.0)]
    gamma = 1.4
    F, u = H.riemann_flux(WL, WR, gamma, velocity=True)
    ok = u.abs() > 0.05
    assert int(ok.sum()) > 3000
    F = [f[ok] for f in F]
    u = u[ok]
    r = F[0] / u
    p = F[1] - F[0] * u
    t1, t2 = F[2] / F[0], F[3] / F[0]
    E = p / (gamma - 1.0) + 0.5 * r * (u * u + t1 * t1 + t2 * t2)
    assert torch.allclose(F[4], u * (E + p), rtol=1e-9, atol=1e-9)
