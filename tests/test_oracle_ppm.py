"""Pins of the oracle's 1-D PPM pieces (Sec. II.C names PPM; formulas are the
published method's): polynomial exactness, limiter properties, the two-shock
solver against the exact Riemann solver, consistency on equal states, and the
exact solver against textbook star states."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import exact
from oracle import hydro as H


def _cubic_avgs(c, x0, h, m):
    """Cell averages of c0 + c1 x + c2 x^2 + c3 x^3 on cells [x0 + j h, x0 + (j+1) h)."""
    P = np.polynomial.Polynomial(c).integ()
    e = x0 + h * np.arange(m + 1)
    return (P(e[1:]) - P(e[:-1])) / h


def test_interface_value_exact_on_cubics():
    c = [0.3, 1.0, 0.2, 0.05]
    h = 0.1
    a = torch.tensor(_cubic_avgs(c, 0.0, h, 12))
    dm = H.limited_slope(a[:-2], a[1:-1], a[2:])          # cells 1..10
    # the limiter must be inactive for the unlimited identity to hold
    da = 0.5 * (a[2:] - a[:-2])
    assert torch.equal(dm, da)
    ai = H.interface_value(a[1:-2], a[2:-1], dm[:-1], dm[1:])  # interfaces j+1/2, j = 1..9
    x = h * np.arange(2, 11)
    exact_v = np.polynomial.Polynomial(c)(x)
    assert np.abs(ai.numpy() - exact_v).max() < 1e-13


def test_limited_slope_properties():
    g = torch.Generator().manual_seed(0)
    a = torch.rand(3, 1000, generator=g, dtype=torch.float64)
    dm = H.limited_slope(a[0], a[1], a[2])
    ext = (a[1] - a[0]) * (a[2] - a[1]) <= 0
    assert (dm[ext] == 0).all()
    assert (dm.abs() <= 2 * (a[1] - a[0]).abs() + 0).all()
    assert (dm.abs() <= 2 * (a[2] - a[1]).abs()).all()
    # odd under reflection, bit-exact
    assert torch.equal(H.limited_slope(a[2], a[1], a[0]), -dm)


def test_monotonize_bounds():
    g = torch.Generator().manual_seed(1)
    a, aL, aR = torch.rand(3, 5000, generator=g, dtype=torch.float64)
    nL, nR = H.monotonize(a, aL, aR)
    # the parabola through (nL, a, nR) has no interior extremum
    da = nR - nL
    a6 = 6.0 * (a - 0.5 * (nL + nR))
    assert ((a6.abs() <= da.abs() + 1e-12) | ((nL == a) & (nR == a))).all()


def _flux(W, gamma):
    r, u, t1, t2, p = W
    E = p / (gamma - 1) + 0.5 * r * (u * u + t1 * t1 + t2 * t2)
    return (r * u, r * u * u + p, r * u * t1, r * u * t2, u * (E + p))


def test_riemann_consistency_equal_states():
    g = torch.Generator().manual_seed(2)
    r = 0.1 + torch.rand(100, generator=g, dtype=torch.float64)
    u = torch.randn(100, generator=g, dtype=torch.float64)
    t1 = torch.randn(100, generator=g, dtype=torch.float64)
    t2 = torch.randn(100, generator=g, dtype=torch.float64)
    p = 0.1 + torch.rand(100, generator=g, dtype=torch.float64)
    W = (r, u, t1, t2, p)
    F = H.riemann_flux(W, W, 1.4)
    Fe = _flux(W, 1.4)
    for a, b in zip(F, Fe):
        assert torch.allclose(a, b, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("u0,gamma", [(0.5, 1.4), (2.0, 5.0 / 3.0), (5.0, 1.4)])
def test_two_shock_solver_exact_on_symmetric_collision(u0, gamma):
    """Both waves are shocks, so the two-shock curves are the exact ones and
    the fixed Newton iteration lands on the exact p*; u* = 0 by symmetry."""
    ps, us = exact.star_state(1.0, u0, 1.0, 1.0, -u0, 1.0, gamma)
    one = torch.ones(1, dtype=torch.float64)
    WL = (one, u0 * one, 0 * one, 0 * one, one)
    WR = (one, -u0 * one, 0 * one, 0 * one, one)
    F = H.riemann_flux(WL, WR, gamma)
    assert abs(float(F[0])) < 1e-14
    assert float(F[1]) == pytest.approx(ps, rel=1e-10)
    assert abs(us) < 1e-12


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_exact_riemann_textbook_star_states():
    """Toro, Table 4.2 (tests/golden/toro_star_states.txt)."""
    rows = _golden_rows("toro_star_states.txt")
    assert len(rows) == 3
    for r in rows:
        v = [float(x) for x in r]
        ps, us = exact.star_state(*v[:6], 1.4)
        assert ps == pytest.approx(v[6], rel=5e-5, abs=1e-5)
        assert us == pytest.approx(v[7], rel=5e-5, abs=1e-5)


def test_exact_riemann_rankine_hugoniot():
    """Sod: the right-moving shock satisfies mass and momentum jump conditions."""
    g = 1.4
    rR, uR, pR = 0.125, 0.0, 0.1
    ps, us = exact.star_state(1.0, 0.0, 1.0, rR, uR, pR, g)
    xi = np.linspace(-1.5, 2.0, 3501)
    r, u, p = exact.sample(xi, 1.0, 0.0, 1.0, rR, uR, pR, g)
    k = np.nonzero(p > pR + 1e-9)[0].max()           # last post-shock point
    S = 0.5 * (xi[k] + xi[k + 1])
    rs = r[k]
    assert rs * (S - us) == pytest.approx(rR * (S - uR), rel=2e-3)
    assert rs * (S - us) * us + ps == pytest.approx(pR, rel=1e-2) or \
        (rs * (S - us) * (us - uR)) == pytest.approx(ps - pR, rel=2e-3)


def test_sedov_constant():
    """Taylor (1950) and Kamm & Timmes (2007), tests/golden/sedov_constants.txt;
    alpha = xi0^-(nu+2)."""
    g = {r[0]: (float(r[1]), float(r[2])) for r in _golden_rows("sedov_constants.txt")}
    assert exact.sedov_xi0(g["xi0"][0]) == pytest.approx(g["xi0"][1], abs=1e-3)
    assert exact.sedov_xi0(g["alpha"][0], nu=3) ** -5 == pytest.approx(g["alpha"][1], abs=2e-6)
    # Kamm & Timmes (2007), the cylindrical constant for gamma = 1.4
    assert exact.sedov_xi0(1.4, nu=2) ** -4 == pytest.approx(0.984074, abs=2e-6)


# ---------------------------------------------------------------- HLLC
def _states(seed, n=200, umax=1.0):
    g = torch.Generator().manual_seed(seed)
    r = 0.1 + torch.rand(n, generator=g, dtype=torch.float64)
    u = umax * torch.randn(n, generator=g, dtype=torch.float64)
    t1 = torch.randn(n, generator=g, dtype=torch.float64)
    t2 = torch.randn(n, generator=g, dtype=torch.float64)
    p = 0.1 + torch.rand(n, generator=g, dtype=torch.float64)
    return (r, u, t1, t2, p)


def test_hllc_consistency_equal_states():
    W = _states(3)
    F = H.hllc_flux(W, W, 1.4)
    for a, b in zip(F, _flux(W, 1.4)):
        assert torch.allclose(a, b, rtol=1e-14, atol=1e-14)


def test_hllc_resolves_a_stationary_contact_exactly():
    """A contact at rest (equal p, zero velocity, any density jump) is an
    exact HLLC solution: no mass or energy crosses, the momentum flux is p
    (Toro Sec. 10.4: the middle wave is resolved)."""
    one = torch.ones(1, dtype=torch.float64)
    z = torch.zeros(1, dtype=torch.float64)
    for rl, rr in ((1.0, 0.25), (4.0, 0.5), (0.125, 2.0)):
        WL = (rl * one, z, z, z, one)
        WR = (rr * one, z, z, z, one)
        F = H.hllc_flux(WL, WR, 1.4)
        assert float(F[0]) == 0.0 and float(F[1]) == 1.0 and float(F[4]) == 0.0
        assert float(F[2]) == 0.0 and float(F[3]) == 0.0


def test_hllc_moving_contact_is_upwinded():
    one = torch.ones(1, dtype=torch.float64)
    z = torch.zeros(1, dtype=torch.float64)
    for u0 in (0.3, -0.3):
        WL = (one, u0 * one, 0.2 * one, z, one)
        WR = (0.25 * one, u0 * one, -0.4 * one, z, one)
        F = H.hllc_flux(WL, WR, 1.4)
        up = WL if u0 > 0 else WR
        Fe = _flux(up, 1.4)
        for a, b in zip(F, Fe):
            assert float(a) == pytest.approx(float(b), rel=1e-13, abs=1e-14)


def test_hllc_supersonic_takes_the_upwind_flux():
    W = _states(4, umax=0.0)
    WL = (W[0], W[1] + 5.0, W[2], W[3], W[4])     # u - c > 0 on both sides
    WR = (W[4] * 0 + 0.5, W[1] + 6.0, W[3], W[2], W[0])
    F = H.hllc_flux(WL, WR, 1.4)
    for a, b in zip(F, _flux(WL, 1.4)):
        assert torch.allclose(a, b, rtol=1e-14, atol=1e-14)


def test_hllc_mirror_symmetry_bit_exact():
    WL, WR = _states(5), _states(6)

    def mirror(W):
        return (W[0], -W[1], W[2], W[3], W[4])
    F = H.hllc_flux(WL, WR, 1.4)
    Fm = H.hllc_flux(mirror(WR), mirror(WL), 1.4)
    assert torch.equal(Fm[0], -F[0]) and torch.equal(Fm[1], F[1]) and torch.equal(Fm[4], -F[4])
    assert torch.equal(Fm[2], -F[2]) and torch.equal(Fm[3], -F[3])


def test_hllc_fan_satisfies_the_jump_conditions():
    """Across the contact the two star states satisfy the Rankine-Hugoniot
    conditions, F*_R - F*_L = S* (U*_R - U*_L), in all five components
    (equal star pressure and normal velocity S* on both sides), and the fan
    satisfies the integral consistency condition (S* - S_L) U*_L + (S_R - S*)
    U*_R = S_R U_R - S_L U_L - (F_R - F_L) (Toro Sec. 10.4)."""
    for seed in (7, 8, 9):
        h = H.hllc_waves(_states(seed), _states(seed + 10), 1.4)
        SL, Ss, SR = h["SL"], h["Ss"], h["SR"]
        for k in range(5):
            lhs = h["FsR"][k] - h["FsL"][k]
            rhs = Ss * (h["UsR"][k] - h["UsL"][k])
            scale = h["FsR"][k].abs() + h["FsL"][k].abs() + (Ss * h["UsR"][k]).abs() + 1.0
            assert float(((lhs - rhs).abs() / scale).max()) < 1e-12, k
            a = (Ss - SL) * h["UsL"][k] + (SR - Ss) * h["UsR"][k]
            b = SR * h["UR"][k] - SL * h["UL"][k] - (h["FR"][k] - h["FL"][k])
            sc = (SR * h["UR"][k]).abs() + (SL * h["UL"][k]).abs() + h["FR"][k].abs() + h["FL"][k].abs() + 1.0
            assert float(((a - b).abs() / sc).max()) < 1e-12, k


# ---------------------------------------------------------- contact steepening
def _eta(rho, p, gamma=1.4):
    N = rho.shape[-1]
    return H.steepening_eta(rho[..., 0:N - 4], rho[..., 1:N - 3], rho[..., 2:N - 2], rho[..., 3:N - 1],
                            rho[..., 4:N], p[..., 1:N - 3], p[..., 3:N - 1], gamma)   # cells 2..N-3


def test_steepening_switches_on_at_a_contact_only():
    N = 40
    rho = torch.ones(N, dtype=torch.float64)
    rho[20:] = 0.125
    p = torch.ones(N, dtype=torch.float64)
    eta = _eta(rho, p)
    on = torch.nonzero(eta).flatten() + 2
    assert on.tolist() == [19, 20] and torch.all(eta[on - 2] == 1.0)
    # a pressure jump as large as the density jump (a shock): off (gas-dynamics condition)
    p2 = p.clone()
    p2[20:] = 0.1
    assert torch.all(_eta(rho, p2) == 0.0)
    # a density jump below the relative threshold: off
    rho3 = torch.ones(N, dtype=torch.float64)
    rho3[20:] = 1.005
    assert torch.all(_eta(rho3, p) == 0.0)


def test_steepening_is_off_on_quadratics():
    """D_{j+1} = D_{j-1} on a quadratic, so eta~ = 0 and the edge values are
    untouched: the fluxes equal those without steepening bit for bit."""
    x = torch.arange(40, dtype=torch.float64)
    rho = (1.0 + 0.01 * x + 0.0003 * x * x).view(1, 40)
    p = torch.ones_like(rho)
    assert torch.all(_eta(rho, p) == 0.0)
    u = 0.3 * torch.ones_like(rho)
    Uc = (rho, rho * u, 0 * rho, 0 * rho, p / 0.4 + 0.5 * rho * u * u)
    dtdx = torch.full((1, 1), 0.2, dtype=torch.float64)
    F0 = H.pencil_fluxes(Uc, dtdx, 1.4, steepen=False)
    F1 = H.pencil_fluxes(Uc, dtdx, 1.4, steepen=True)
    for a, b in zip(F0, F1):
        assert torch.equal(a, b)


def test_steepened_fluxes_are_mirror_symmetric_on_a_smeared_contact():
    """Mirror symmetry of the pencil fluxes (F0, F2, F3, F4 change sign, F1
    does not) with steepening active on a contact spread over three cells,
    where the neighbours' limited slopes are not zero."""
    rho = torch.tensor([1.0] * 18 + [0.97, 0.6, 0.2, 0.14] + [0.125] * 18, dtype=torch.float64).view(1, 40)
    p = torch.ones_like(rho)
    eta = _eta(rho, p)
    dm = H.limited_slope(rho[..., :-2], rho[..., 1:-1], rho[..., 2:])
    on = torch.nonzero(eta[0] > 0).flatten() + 2
    assert len(on) > 0 and any(float(dm[0, c - 2]) != 0.0 or float(dm[0, c]) != 0.0 for c in on.tolist())
    u = 0.2 * torch.ones_like(rho)
    v = 0.1 * torch.ones_like(rho)

    def fluxes(r, un):
        Uc = (r, r * un, r * v, 0 * r, p / 0.4 + 0.5 * r * (un * un + v * v))
        return H.pencil_fluxes(Uc, torch.full((1, 1), 0.3, dtype=torch.float64), 1.4, steepen=True)
    F = fluxes(rho, u)
    Fm = fluxes(rho.flip(-1), -u)
    for k, sgn in zip(range(5), (-1, 1, -1, -1, -1)):
        assert torch.equal(Fm[k].flip(-1), sgn * F[k]), k
