"""Pins of the oracle's 1-D PPM pieces (Sec. II.C names PPM; formulas are the
published method's): polynomial exactness, limiter properties, the two-shock
solver against the exact Riemann solver, consistency on equal states, and the
exact solver against textbook star states."""
import math

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


def test_exact_riemann_textbook_star_states():
    # Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", Table 4.2
    cases = [((1.0, 0.0, 1.0, 0.125, 0.0, 0.1), (0.30313, 0.92745)),
             ((1.0, -2.0, 0.4, 1.0, 2.0, 0.4), (0.00189, 0.0)),
             ((1.0, 0.0, 1000.0, 1.0, 0.0, 0.01), (460.894, 19.5975))]
    for args, (p, u) in cases:
        ps, us = exact.star_state(*args, 1.4)
        assert ps == pytest.approx(p, rel=5e-5, abs=1e-5)
        assert us == pytest.approx(u, rel=5e-5, abs=1e-5)


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
    # Taylor (1950): R = 1.033 (E t^2/rho)^(1/5) for gamma = 1.4
    assert exact.sedov_xi0(1.4) == pytest.approx(1.033, abs=1e-3)
    # Kamm & Timmes (2007), energy constants alpha = xi0^-(nu+2) for gamma = 1.4
    assert exact.sedov_xi0(1.4, nu=3) ** -5 == pytest.approx(0.851072, abs=2e-6)
    assert exact.sedov_xi0(1.4, nu=2) ** -4 == pytest.approx(0.984074, abs=2e-6)
