"""Plain FP64 oracle of one Enzo-P/Cello hydro step over the leaves of an
array-of-octrees mesh.  TEST INFRASTRUCTURE ONLY: used by tests/, by the
smoke check and by the CPU-baseline leg of the benchmark, never by the
product library.

What the paper fixes (Sec. II.B, II.C): leaf Blocks carry the fields; a ghost
layer of configurable width around each Block is refreshed from neighbouring
Blocks before a Method runs (Sec. II.B, Fig. 4); Refine / Restrict / Prolong
plug-ins move data between levels (Sec. II.B); the hydro Method is a modified
piecewise parabolic method (PPM, Colella & Woodward 1984; Bryan et al. 1995)
(Sec. II.C).  The paper prints none of the formulas, so every formula below is
a reading of the named published method, stated in the docstrings.  The
code is vectorised torch float64 on the CPU: every
elementwise operation is written out in the stated order (no fused
multiply-add, no reassociation), so a reader can check it term by term.

Layout: U[B, 5, N, N, N] float64, leaves in mesh order, conserved fields
(rho, rho*u, rho*v, rho*w, E), cells indexed [z, y, x] with N = n + 2g; with
the dual-energy formalism (Desc.dual_energy) U[B, 6, N, N, N], the sixth
field the internal energy density rho*e (see dual_energy_sync below).

Parity pins (tests/test_oracle_*.py): uniform-state invariance, mirror
symmetry, conservation on periodic AMR meshes, all-one-level AMR equal to a
single uniform block, Sod against the exact Riemann solution, interface
formula exact on cubics, two-shock solver exact on symmetric collisions,
prolongation/restriction identities, CFL closed form, brute-force flags.
"""
from __future__ import annotations

import numpy as np
import torch

from .mesh import FINE, OUTFLOW, PERIODIC, Mesh, neighbour_table  # noqa: F401

RHO_FLOOR = 1e-10
P_FLOOR = 1e-20
EPS_SHOCK = 0.33     # CW84 shock-detector threshold on the relative pressure jump
OMEGA1 = 0.75        # CW84 flattening: ratio offset
OMEGA2 = 10.0        # CW84 flattening: ratio slope
N_RIEMANN = 5        # fixed Newton iterations of the two-shock solver, no early exit
EPS_STEEP = 0.01     # CW84 contact steepening: least relative density jump
ETA1, ETA2 = 20.0, 0.05   # CW84 contact steepening: eta = clamp(ETA1 (eta~ - ETA2), 0, 1)
K0_STEEP = 0.1       # CW84 gas-dynamics condition: steepen where the density jump dominates
DE_ETA1 = 1e-3       # dual energy: pressure from E where E - ke > DE_ETA1 E, else from rho e
DE_ETA2 = 0.1        # dual energy: rho e reset to E - ke after a sweep where E - ke > DE_ETA2 E
SIXTH = 1.0 / 6.0
TWO_THIRDS = 2.0 / 3.0
GHOSTS = 4           # the PPM stencil below reaches 4 cells on each side

# conserved component order seen by a sweep along each axis:
# (density, normal momentum, transverse momentum 1, transverse momentum 2, E,
# and rho e with the dual-energy formalism)
AXIS_COMPONENTS = {0: (0, 1, 2, 3, 4, 5), 1: (0, 2, 1, 3, 4, 5), 2: (0, 3, 1, 2, 4, 5)}
AXIS_DIM = {0: 4, 1: 3, 2: 2}   # tensor dim of an axis in U[B, 5, z, y, x]


# ----------------------------------------------------------------- 1-D PPM
def ieee_sqrt(x):
    """Correctly rounded float64 square root.  torch's vectorised CPU sqrt
    is not always correctly rounded (1 ulp off for about 1% of inputs); the
    value here is numpy's IEEE sqrt, the gradient torch's."""
    s = torch.sqrt(x)
    exact = torch.from_numpy(np.sqrt(x.detach().cpu().numpy())).to(s.device)
    return s + (exact - s).detach()


def primitives(rho_c, mn, mt1, mt2, E, gamma, rhoe=None):
    """Conserved -> primitive (rho, u_n, u_t1, u_t2, p) with density and
    pressure floors.  Kinetic energy 0.5*rho*(u_n^2 + (u_t1^2 + u_t2^2)).
    With the dual-energy formalism (rhoe given, Bryan et al. 1995): the
    pressure comes from the internal energy E - ke where E - ke > DE_ETA1 E,
    else from rho e, and the specific internal energy e = rho e / rho is a
    sixth primitive."""
    rho = torch.clamp_min(rho_c, RHO_FLOOR)
    un = mn / rho
    ut1 = mt1 / rho
    ut2 = mt2 / rho
    ke = (0.5 * rho) * (un * un + (ut1 * ut1 + ut2 * ut2))
    if rhoe is None:
        p = torch.clamp_min((gamma - 1.0) * (E - ke), P_FLOOR)
        return rho, un, ut1, ut2, p
    eint = E - ke
    p = torch.clamp_min((gamma - 1.0) * torch.where(eint > DE_ETA1 * E, eint, rhoe), P_FLOOR)
    return rho, un, ut1, ut2, p, rhoe / rho


def dual_energy_sync(rho_c, mn, mt1, mt2, E, rhoe):
    """Dual-energy synchronisation after a sweep's update (Bryan et al.
    1995): where the internal energy from the total energy, E - ke (ke as in
    primitives, from the updated state), exceeds DE_ETA2 E it replaces rho e;
    elsewhere rho e keeps its own update."""
    rho = torch.clamp_min(rho_c, RHO_FLOOR)
    un = mn / rho
    ut1 = mt1 / rho
    ut2 = mt2 / rho
    ke = (0.5 * rho) * (un * un + (ut1 * ut1 + ut2 * ut2))
    eint = E - ke
    return torch.where(eint > DE_ETA2 * E, eint, rhoe)


def limited_slope(am, a0, ap):
    """CW84 monotonised centred slope: 0.5*(a+ - a-), limited to twice the
    one-sided differences, zero at a local extremum."""
    dl = a0 - am
    dr = ap - a0
    da = 0.5 * (ap - am)
    m = torch.minimum(torch.abs(da), torch.minimum(2.0 * torch.abs(dl), 2.0 * torch.abs(dr)))
    return torch.where(dl * dr > 0.0, torch.copysign(m, da), torch.zeros_like(da))


def interface_value(a0, a1, dm0, dm1):
    """CW84 interface value between cells j and j+1 in limited form:
    0.5*(a_j + a_j+1) - (dm_j+1 - dm_j)/6.  With unlimited slopes this is the
    fourth-order (7/12, -1/12) interpolant, exact for cell averages of cubics."""
    return 0.5 * (a0 + a1) - (dm1 - dm0) * SIXTH


def flatten_tilde(pm2, pm1, pp1, pp2, um1, up1):
    """CW84 shock detector: nonzero only across a compressive pressure jump
    larger than EPS_SHOCK relative; 10*(dp1/dp2 - 0.75) clipped to [0, 1]."""
    dp1 = pp1 - pm1
    dp2 = pp2 - pm2
    shock = (torch.abs(dp1) > EPS_SHOCK * torch.minimum(pp1, pm1)) & (um1 - up1 > 0.0) & (dp2 != 0.0)
    ratio = dp1 / torch.where(dp2 != 0.0, dp2, torch.ones_like(dp2))
    ft = torch.clamp_min(torch.clamp_max(OMEGA2 * (ratio - OMEGA1), 1.0), 0.0)
    return torch.where(shock, ft, torch.zeros_like(ft))


def monotonize(a, aL, aR):
    """CW84 monotonicity constraints on the parabola of one cell."""
    ext = (aR - a) * (a - aL) <= 0.0
    da = aR - aL
    dm = a - 0.5 * (aL + aR)
    t1 = da * dm
    t2 = (da * da) * SIXTH
    nL = torch.where(ext, a, torch.where(t1 > t2, 3.0 * a - 2.0 * aR, aL))
    nR = torch.where(ext, a, torch.where(-t2 > t1, 3.0 * a - 2.0 * aL, aR))
    return nL, nR


def edge_avg_right(aL, aR, a6, sigma):
    """Average of the cell parabola over the last sigma of the cell (CW84)."""
    da = aR - aL
    return aR - (0.5 * sigma) * (da - (1.0 - TWO_THIRDS * sigma) * a6)


def edge_avg_left(aL, aR, a6, sigma):
    """Average of the cell parabola over the first sigma of the cell (CW84)."""
    da = aR - aL
    return aL + (0.5 * sigma) * (da + (1.0 - TWO_THIRDS * sigma) * a6)


def trace(W, aL, aR, dtdx, gamma):
    """Characteristic tracing of one cell to its two edges at the half step.

    Waves u-c, u, u+c with the left/right eigenvectors of the primitive
    (rho, u, p) system at the cell centre.  Right edge: reference state = the
    average seen by the fastest wave moving right (or aR if none does); every
    other wave moving right subtracts its projection l.(ref - avg) along its
    right eigenvector.  Left edge mirrors it.  Transverse velocities ride the
    entropy wave, and so does the specific internal energy e of the
    dual-energy formalism (a sixth component, advected).  Returns (state at
    the left edge, state at the right edge), each (rho, u_n, u_t1, u_t2, p)
    [+ e], floored."""
    nq = len(W)
    rho, un, p = W[0], W[1], W[4]
    csq = (gamma * p) / rho
    c = ieee_sqrt(csq)
    a6 = [6.0 * (W[q] - 0.5 * (aL[q] + aR[q])) for q in range(nq)]
    lm, l0, lp = un - c, un, un + c
    half_rho_c = (0.5 * rho) / c
    half_inv_csq = 0.5 / csq
    c_rho = c / rho
    zero = torch.zeros_like(un)

    # right edge: waves with lambda > 0
    sp, s0, sm = lp * dtdx, l0 * dtdx, lm * dtdx
    ref = [torch.where(lp > 0.0, edge_avg_right(aL[q], aR[q], a6[q], sp), aR[q]) for q in range(nq)]
    bm = torch.where(lm > 0.0,
                     (ref[4] - edge_avg_right(aL[4], aR[4], a6[4], sm)) * half_inv_csq
                     - (ref[1] - edge_avg_right(aL[1], aR[1], a6[1], sm)) * half_rho_c, zero)
    b0 = torch.where(l0 > 0.0,
                     (ref[0] - edge_avg_right(aL[0], aR[0], a6[0], s0))
                     - (ref[4] - edge_avg_right(aL[4], aR[4], a6[4], s0)) / csq, zero)
    r_rho = torch.clamp_min(ref[0] - (b0 + bm), RHO_FLOOR)
    r_un = ref[1] + c_rho * bm
    r_p = torch.clamp_min(ref[4] - csq * bm, P_FLOOR)
    r_t1 = torch.where(l0 > 0.0, edge_avg_right(aL[2], aR[2], a6[2], s0), ref[2])
    r_t2 = torch.where(l0 > 0.0, edge_avg_right(aL[3], aR[3], a6[3], s0), ref[3])
    r_e = [torch.where(l0 > 0.0, edge_avg_right(aL[q], aR[q], a6[q], s0), ref[q]) for q in range(5, nq)]

    # left edge: waves with lambda < 0
    tm, t0, tp = -lm * dtdx, -l0 * dtdx, -lp * dtdx
    ref = [torch.where(lm < 0.0, edge_avg_left(aL[q], aR[q], a6[q], tm), aL[q]) for q in range(nq)]
    bp = torch.where(lp < 0.0,
                     (ref[4] - edge_avg_left(aL[4], aR[4], a6[4], tp)) * half_inv_csq
                     + (ref[1] - edge_avg_left(aL[1], aR[1], a6[1], tp)) * half_rho_c, zero)
    b0 = torch.where(l0 < 0.0,
                     (ref[0] - edge_avg_left(aL[0], aR[0], a6[0], t0))
                     - (ref[4] - edge_avg_left(aL[4], aR[4], a6[4], t0)) / csq, zero)
    l_rho = torch.clamp_min(ref[0] - (b0 + bp), RHO_FLOOR)
    l_un = ref[1] - c_rho * bp
    l_p = torch.clamp_min(ref[4] - csq * bp, P_FLOOR)
    l_t1 = torch.where(l0 < 0.0, edge_avg_left(aL[2], aR[2], a6[2], t0), ref[2])
    l_t2 = torch.where(l0 < 0.0, edge_avg_left(aL[3], aR[3], a6[3], t0), ref[3])
    l_e = [torch.where(l0 < 0.0, edge_avg_left(aL[q], aR[q], a6[q], t0), ref[q]) for q in range(5, nq)]
    return (l_rho, l_un, l_t1, l_t2, l_p, *l_e), (r_rho, r_un, r_t1, r_t2, r_p, *r_e)


def riemann_flux(WL, WR, gamma, velocity=False):
    """CW84 two-shock approximate Riemann solver with N_RIEMANN fixed Newton
    steps on p* (shock curves on both sides, derivative Z = 2W^3/(W^2+C^2)),
    u* = Z-weighted mean, sampled at x/t = 0 (u* >= 0 takes the left side);
    inside a rarefaction the state is interpolated linearly between the head
    and tail speeds.  Returns the five fluxes (rho, m_n, m_t1, m_t2, E); with
    a sixth component e (dual energy) also the flux of rho e, the mass flux
    times the e of the sampled side (e rides with the transverse
    velocities).  velocity=True returns (fluxes, u) with u the normal
    velocity of the sampled state."""
    rL, uL, t1L, t2L, pL = WL[:5]
    rR, uR, t1R, t2R, pR = WR[:5]
    g1 = (gamma + 1.0) / (2.0 * gamma)
    CL = ieee_sqrt((gamma * pL) * rL)
    CR = ieee_sqrt((gamma * pR) * rR)
    ps = ((CR * pL + CL * pR) + (CL * CR) * (uL - uR)) / (CL + CR)
    ps = torch.clamp_min(ps, P_FLOOR)

    def curves(ps):
        WLs = CL * ieee_sqrt(1.0 + g1 * (ps / pL - 1.0))
        WRs = CR * ieee_sqrt(1.0 + g1 * (ps / pR - 1.0))
        uLs = uL - (ps - pL) / WLs
        uRs = uR + (ps - pR) / WRs
        ZL = ((2.0 * WLs) * WLs) * WLs / (WLs * WLs + CL * CL)
        ZR = ((2.0 * WRs) * WRs) * WRs / (WRs * WRs + CR * CR)
        return WLs, WRs, uLs, uRs, ZL, ZR

    for _ in range(N_RIEMANN):
        _, _, uLs, uRs, ZL, ZR = curves(ps)
        ps = torch.clamp_min(ps - ((ZL * ZR) * (uRs - uLs)) / (ZL + ZR), P_FLOOR)
    WLs, WRs, uLs, uRs, ZL, ZR = curves(ps)
    us = (ZL * uLs + ZR * uRs) / (ZL + ZR)

    left = us >= 0.0
    rs = torch.where(left, rL, rR)
    u_s = torch.where(left, uL, uR)
    p_s = torch.where(left, pL, pR)
    W_s = torch.where(left, WLs, WRs)
    t1 = torch.where(left, t1L, t1R)
    t2 = torch.where(left, t2L, t2R)
    v_s = torch.where(left, -uL, uR)        # outward normal velocity of the sampled side
    v_star = torch.where(left, -us, us)
    tau = 1.0 / rs - (ps - p_s) / (W_s * W_s)
    rstar = torch.where(tau > 0.0, 1.0 / torch.where(tau > 0.0, tau, torch.ones_like(tau)),
                        torch.full_like(tau, RHO_FLOOR))
    rstar = torch.clamp_min(rstar, RHO_FLOOR)
    c_s = ieee_sqrt((gamma * p_s) / rs)
    c_star = ieee_sqrt((gamma * ps) / rstar)
    shock = ps > p_s
    head = torch.where(shock, v_s + W_s / rs, v_s + c_s)
    tail = torch.where(shock, head, v_star + c_star)
    orig = head <= 0.0
    star = (~orig) & (tail > 0.0)
    den = head - tail
    w = head / torch.where(orig | star, torch.ones_like(den), den)
    fan_r = rs + w * (rstar - rs)
    fan_u = u_s + w * (us - u_s)
    fan_p = p_s + w * (ps - p_s)
    r = torch.where(orig, rs, torch.where(star, rstar, fan_r))
    u = torch.where(orig, u_s, torch.where(star, us, fan_u))
    p = torch.where(orig, p_s, torch.where(star, ps, fan_p))

    inv_gm1 = 1.0 / (gamma - 1.0)
    f0 = r * u
    f1 = f0 * u + p
    f2 = f0 * t1
    f3 = f0 * t2
    E = p * inv_gm1 + (0.5 * r) * (u * u + (t1 * t1 + t2 * t2))
    f4 = u * (E + p)
    F = (f0, f1, f2, f3, f4)
    if len(WL) > 5:
        F = F + (f0 * torch.where(left, WL[5], WR[5]),)
    return (F, u) if velocity else F


def hllc_waves(WL, WR, gamma):
    """The HLLC wave fan (Toro, Spruce & Speares 1994; Toro, "Riemann Solvers
    and Numerical Methods for Fluid Dynamics", 3rd ed., Sec. 10.4) of left
    and right primitive states (rho, u_n, u_t1, u_t2, p): wave-speed bounds
    of Davis, S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R +
    c_R); contact speed S* = (p_R - p_L + m_L u_L - m_R u_R) / (m_L - m_R)
    with m_K = rho_K (S_K - u_K) (Toro eq. 10.37); star states U*_K = m_K /
    (S_K - S*) (1, S*, v_K, w_K, E_K / rho_K + (S* - u_K)(S* + p_K / m_K))
    (eq. 10.39) and star fluxes F*_K = F_K + S_K (U*_K - U_K) (eq. 10.38).
    A sixth component e (dual energy) is passive like v and w: conserved
    rho e, flux rho u e, star value m_K / (S_K - S*) e_K.  Returns a dict of
    the speeds, the side states U, fluxes F and the star states and
    fluxes."""
    inv_gm1 = 1.0 / (gamma - 1.0)

    def side(W):
        r, u, v, w, p = W[:5]
        c = ieee_sqrt((gamma * p) / r)
        E = p * inv_gm1 + (0.5 * r) * (u * u + (v * v + w * w))
        f0 = r * u
        F = (f0, f0 * u + p, f0 * v, f0 * w, u * (E + p)) + tuple(f0 * e for e in W[5:])
        Uc = (r, r * u, r * v, r * w, E) + tuple(r * e for e in W[5:])
        return c, E, F, Uc

    rL, uL, vL, wL, pL = WL[:5]
    rR, uR, vR, wR, pR = WR[:5]
    cL, EL, FL, UL = side(WL)
    cR, ER, FR, UR = side(WR)
    SL = torch.minimum(uL - cL, uR - cR)
    SR = torch.maximum(uL + cL, uR + cR)
    mL = rL * (SL - uL)
    mR = rR * (SR - uR)
    Ss = ((pR - pL) + (mL * uL - mR * uR)) / (mL - mR)

    def star(S, m, r, u, v, w, p, E, F, Uc, extra):
        fac = m / (S - Ss)
        Us = ((fac, fac * Ss, fac * v, fac * w, fac * (E / r + (Ss - u) * (Ss + p / m)))
              + tuple(fac * e for e in extra))
        return Us, tuple(Fk + S * (Usk - Uk) for Fk, Usk, Uk in zip(F, Us, Uc))

    UsL, FsL = star(SL, mL, rL, uL, vL, wL, pL, EL, FL, UL, WL[5:])
    UsR, FsR = star(SR, mR, rR, uR, vR, wR, pR, ER, FR, UR, WR[5:])
    return dict(SL=SL, SR=SR, Ss=Ss, UL=UL, UR=UR, FL=FL, FR=FR, UsL=UsL, UsR=UsR, FsL=FsL, FsR=FsR)


def hllc_flux(WL, WR, gamma, velocity=False):
    """HLLC interface flux, an alternative to the two-shock flux of the PPM
    sweep: the flux of the region of the fan (hllc_waves) holding x/t = 0,
    F_L if S_L >= 0, F*_L if S* >= 0, F*_R if S_R > 0, else F_R.  Returns
    the five fluxes (rho, m_n, m_t1, m_t2, E) (six with dual energy);
    velocity=True returns (fluxes, u) with u the normal velocity of that
    region's state: u_L, S*, S*, u_R."""
    h = hllc_waves(WL, WR, gamma)
    SL, Ss, SR = h["SL"], h["Ss"], h["SR"]
    out = []
    for k in range(len(WL)):
        out.append(torch.where(SL >= 0.0, h["FL"][k],
                               torch.where(Ss >= 0.0, h["FsL"][k],
                                           torch.where(SR > 0.0, h["FsR"][k], h["FR"][k]))))
    if not velocity:
        return tuple(out)
    u = torch.where(SL >= 0.0, WL[1], torch.where(Ss >= 0.0, Ss, torch.where(SR > 0.0, Ss, WR[1])))
    return tuple(out), u


RIEMANN = {"two-shock": riemann_flux, "hllc": hllc_flux}


def steepening_eta(rm2, rm1, r0, rp1, rp2, pm1, pp1, gamma):
    """Contact-steepening weight of a cell (Colella & Woodward 1984, Sec. 1,
    eqs. 1.14-1.17 on a uniform grid, and the gas-dynamics condition of
    Sec. 3, eq. 3.2) from the densities of cells j-2 .. j+2 and the pressures
    of cells j-1, j+1: with D_c = rho_{c+1} - 2 rho_c + rho_{c-1},
    eta~ = -(D_{j+1} - D_{j-1}) / (6 (rho_{j+1} - rho_{j-1})), set to 0 where
    D_{j+1} D_{j-1} > 0, where |rho_{j+1} - rho_{j-1}| < EPS_STEEP
    min(|rho_{j+1}|, |rho_{j-1}|), or where gamma K0 |rho_{j+1} - rho_{j-1}| /
    min(rho_{j+1}, rho_{j-1}) < |p_{j+1} - p_{j-1}| / min(p_{j+1}, p_{j-1});
    eta = clamp(ETA1 (eta~ - ETA2), 0, 1)."""
    Dm = (r0 - 2.0 * rm1) + rm2
    Dp = (rp2 - 2.0 * rp1) + r0
    drho = rp1 - rm1
    off = ((Dp * Dm > 0.0)
           | (drho.abs() - EPS_STEEP * torch.minimum(rp1.abs(), rm1.abs()) < 0.0)
           | (((gamma * K0_STEEP) * drho.abs()) / torch.minimum(rp1, rm1)
              < (pp1 - pm1).abs() / torch.minimum(pp1, pm1)))
    safe = torch.where(off, torch.ones_like(drho), drho)
    eta_t = torch.where(off, torch.zeros_like(drho), -(Dp - Dm) / (6.0 * safe))
    return torch.clamp(torch.clamp(ETA1 * (eta_t - ETA2), max=1.0), min=0.0)


def pencil_fluxes(Uc, dtdx, gamma, riemann="two-shock", steepen=False, dual=False):
    """Fluxes at the n+1 interfaces between cells c and c+1, c = 3 .. N-5, of
    pencils of length N = n + 8 (last tensor dim).  Uc = (rho, m_n, m_t1,
    m_t2, E) tensors; riemann names the interface solver; steepen applies
    contact steepening to the density edge values (before flattening and the
    monotonicity constraints, as in CW84).  dual: Uc has a sixth tensor rho e
    (dual-energy formalism); the return is then (fluxes, u, p) with u the
    normal velocity of the interface states and p the cell pressures
    (primitives), both for the source term of the internal energy."""
    N = Uc[0].shape[-1]
    W = primitives(*Uc[:5], gamma, rhoe=Uc[5] if dual else None)
    p, un = W[4], W[1]
    dm = [limited_slope(a[..., :-2], a[..., 1:-1], a[..., 2:]) for a in W]           # cells 1..N-2
    ai = [0.5 * (a[..., 1:N - 2] + a[..., 2:N - 1]) - (d[..., 1:] - d[..., :-1]) * SIXTH
          for a, d in zip(W, dm)]                                                        # j+1/2, j=1..N-3
    ft = flatten_tilde(p[..., 0:N - 4], p[..., 1:N - 3], p[..., 3:N - 1], p[..., 4:N],
                       un[..., 1:N - 3], un[..., 3:N - 1])                                # cells 2..N-3
    s = p[..., 4:N - 2] - p[..., 2:N - 4]                                                  # cells 3..N-4
    fj, fm, fp = ft[..., 1:N - 5], ft[..., 0:N - 6], ft[..., 2:N - 4]
    f = torch.where(s > 0.0, torch.maximum(fj, fm), torch.where(s < 0.0, torch.maximum(fj, fp), fj))
    Wc = [a[..., 3:N - 3] for a in W]
    aL, aR = [], []
    for q in range(len(W)):
        l = ai[q][..., 1:N - 5]
        r = ai[q][..., 2:N - 4]
        if steepen and q == 0:                                                              # cells 3..N-4
            rho = W[0]
            eta = steepening_eta(rho[..., 1:N - 5], rho[..., 2:N - 4], rho[..., 3:N - 3], rho[..., 4:N - 2],
                                 rho[..., 5:N - 1], p[..., 2:N - 4], p[..., 4:N - 2], gamma)
            dmm, dmp = dm[0][..., 1:N - 5], dm[0][..., 3:N - 3]                             # slopes of j-1, j+1
            l = l * (1.0 - eta) + (rho[..., 2:N - 4] + 0.5 * dmm) * eta
            r = r * (1.0 - eta) + (rho[..., 4:N - 2] - 0.5 * dmp) * eta
        l = f * Wc[q] + (1.0 - f) * l
        r = f * Wc[q] + (1.0 - f) * r
        l, r = monotonize(Wc[q], l, r)
        aL.append(l)
        aR.append(r)
    Wm, Wp = trace(Wc, aL, aR, dtdx, gamma)        # cells 3..N-4
    left = [x[..., 0:N - 7] for x in Wp]
    right = [x[..., 1:N - 6] for x in Wm]
    if not dual:
        return RIEMANN[riemann](left, right, gamma)
    F, u = RIEMANN[riemann](left, right, gamma, velocity=True)
    return F, u, p


# ------------------------------------------------------------------ sweeps
def dx_of_leaves(mesh: Mesh):
    d = mesh.desc
    return torch.tensor([d.dx(int(L)) for L in mesh.leaves[:, 0]], dtype=torch.float64)


def dtdx_of_leaves(mesh: Mesh, dt: float):
    """dt/dx per leaf, each a correctly rounded float64 quotient (torch would
    evaluate a scalar over a tensor as a reciprocal times the scalar)."""
    d = mesh.desc
    return torch.tensor([dt / d.dx(int(L)) for L in mesh.leaves[:, 0]], dtype=torch.float64)


def sweep(U, mesh: Mesh, axis: int, dt: float, rows):
    """One directional PPM sweep of every leaf.  rows = ((lo, hi), (lo, hi))
    ranges of the two transverse tensor dims (in their U order) whose pencils
    are updated; cells g..g+n-1 along the axis are updated in place.
    Returns (U, faces) with faces = (F at interface g-1/2, F at g+n-1/2) on
    interior rows, each [B, nf, n, n] indexed [t2, t1] (t1 < t2 axes).

    Dual-energy formalism (Bryan et al. 1995): rho e is updated by its flux
    difference and by the compression term of the internal-energy equation,
    rho e <- (rho e - (dt/dx) (F+ - F-)) - ((dt/dx) p) (u+ - u-), p the
    cell's pressure from primitives and u+-, the normal velocities of the
    interface states on its two faces; then dual_energy_sync on the updated
    cells."""
    d = mesh.desc
    n, g = d.n, d.ghosts
    assert g == GHOSTS
    nf = d.nf
    B = U.shape[0]
    dim = AXIS_DIM[axis]
    comp = AXIS_COMPONENTS[axis]
    V = U.movedim(dim, -1)
    dtdx = dtdx_of_leaves(mesh, dt).view(B, 1, 1, 1)
    F = pencil_fluxes([V[:, comp[q]] for q in range(nf)], dtdx, d.gamma, d.riemann, d.steepen, d.dual_energy)
    if d.dual_energy:
        F, uf, pc = F
    (a0, a1), (b0, b1) = rows
    V2 = V.clone()
    for q in range(nf):
        Fq = F[q][:, a0:a1, b0:b1]
        V2[:, comp[q], a0:a1, b0:b1, g:g + n] = (V[:, comp[q], a0:a1, b0:b1, g:g + n]
                                                - dtdx * (Fq[..., 1:] - Fq[..., :-1]))
    if d.dual_energy:
        uq = uf[:, a0:a1, b0:b1]
        pq = pc[:, a0:a1, b0:b1, g:g + n]
        cell = (slice(None), slice(a0, a1), slice(b0, b1), slice(g, g + n))
        e = V2[:, 5][cell] - (dtdx * pq) * (uq[..., 1:] - uq[..., :-1])
        V2[:, 5][cell] = dual_energy_sync(*(V2[:, comp[q]][cell] for q in range(5)), e)
    inv = [0] * nf
    for q in range(nf):
        inv[comp[q]] = q
    lo = torch.stack([F[inv[f]][:, g:g + n, g:g + n, 0] for f in range(nf)], 1)
    hi = torch.stack([F[inv[f]][:, g:g + n, g:g + n, n] for f in range(nf)], 1)
    return V2.movedim(-1, dim), (lo, hi)


def sweep_order(cycle: int):
    """x, y, z on even cycles and z, y, x on odd ones (Strang-type alternation)."""
    return (0, 1, 2) if cycle % 2 == 0 else (2, 1, 0)


def transverse_rows(mesh: Mesh, axis: int, swept):
    """Rows updated by a sweep: a transverse axis already swept this step
    needs interior rows only, one not yet swept needs all N rows (the later
    sweeps read its ghost rows)."""
    n, g = mesh.desc.n, mesh.desc.ghosts
    N = n + 2 * g
    dims = [a for a in (2, 1, 0) if a != axis]      # transverse axes in U dim order (z, y, x)
    return tuple((g, g + n) if a in swept else (0, N) for a in dims)


# ----------------------------------------------------------- ghost refresh
def _bc(mesh: Mesh, M: int, axis: int, v):
    """Apply the physical boundary to level-M global cell indices: periodic
    wraps, outflow clamps to the nearest interior cell."""
    ncell = (mesh.desc.root[axis] << M) * mesh.desc.n
    if mesh.desc.bc[axis] == PERIODIC:
        return np.mod(v, ncell)
    return np.clip(v, 0, ncell - 1)


class RefreshPlan:
    """Gather plan of the ghost refresh for one mesh.

    For a ghost cell of a leaf at level L, with global level-L cell index X
    after the boundary rule, the value is that of the level-L cell X:
      * covered by a level-L leaf: copy;
      * covered by level-L+1 leaves: restriction, the mean of its 8 children
        summed in (dz, dy, dx) lexicographic order, times 0.125;
      * covered by a level-L-1 leaf: conservative linear prolongation of the
        parent cell C: U_f = U_C + 0.25*((sx*Dx + sy*Dy) + sz*Dz) with
        s = +1 for the upper child, D_d = minmod(U_C - U_C-e_d, U_C+e_d - U_C);
        the level-L-1 neighbours C+-e_d (boundary rule at level L-1) are copied
        from a level-L-1 leaf, restricted from level-L leaves or injected from
        the level-L-2 leaf that covers them.
    The sources are always leaf interiors, so the refresh has no ordering.

    dest: optional list of leaf indices whose ghosts the plan fills (all
    leaves by default); sources may still be any leaf of the mesh."""

    def __init__(self, mesh: Mesh, dest=None):
        d = mesh.desc
        n, g = d.n, d.ghosts
        N = n + 2 * g
        self.N3 = N ** 3
        self.nf = nf = d.nf
        maps = mesh.maps()
        zz, yy, xx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        inner = ((xx >= g) & (xx < g + n) & (yy >= g) & (yy < g + n) & (zz >= g) & (zz < g + n))
        gz, gy, gx = zz[~inner], yy[~inner], xx[~inner]
        gcell = (gz * N + gy) * N + gx
        N3 = self.N3

        def flat(b, z, y, x):
            return b * nf * N3 + (z * N + y) * N + x

        def leaf_at(M, X, Y, Z):
            return maps[M][Z // n, Y // n, X // n]

        copy_d, copy_s = [], []
        rst_d, rst_s = [], []
        pro_d, pro_c, pro_sg, pro_nb, pro_mode = [], [], [], [], []

        def restrict_src(M, X, Y, Z):
            """8 children (level M+1) of level-M cells, order (dz, dy, dx)."""
            srcs = []
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        x2, y2, z2 = 2 * X + dx, 2 * Y + dy, 2 * Z + dz
                        f = leaf_at(M + 1, x2, y2, z2)
                        assert (f >= 0).all()
                        srcs.append(flat(f, z2 % n + g, y2 % n + g, x2 % n + g))
            return np.stack(srcs, -1)

        def value0(M, X, Y, Z):
            """Sources of level-M cells for prolongation slopes:
            returns (idx[k, 8], mode[k]) mode 0 single source, 1 mean of 8."""
            m = leaf_at(M, X, Y, Z)
            idx = np.zeros(X.shape + (8,), dtype=np.int64)
            mode = np.zeros(X.shape, dtype=np.int64)
            s = m >= 0
            idx[s, 0] = flat(m[s], Z[s] % n + g, Y[s] % n + g, X[s] % n + g)
            f = m == -1
            if f.any():
                idx[f] = restrict_src(M, X[f], Y[f], Z[f])
                mode[f] = 1
            c = m == -2
            if c.any():
                Xc, Yc, Zc = X[c] // 2, Y[c] // 2, Z[c] // 2
                cc = leaf_at(M - 1, Xc, Yc, Zc)
                assert (cc >= 0).all()
                idx[c, 0] = flat(cc, Zc % n + g, Yc % n + g, Xc % n + g)
            return idx, mode

        for b in (range(mesh.n_leaves) if dest is None else dest):
            L, bi, bj, bk = (int(v) for v in mesh.leaves[b])
            X = _bc(mesh, L, 0, bi * n + gx - g)
            Y = _bc(mesh, L, 1, bj * n + gy - g)
            Z = _bc(mesh, L, 2, bk * n + gz - g)
            dst = b * nf * N3 + gcell
            m = leaf_at(L, X, Y, Z)
            s = m >= 0
            copy_d.append(dst[s])
            copy_s.append(flat(m[s], Z[s] % n + g, Y[s] % n + g, X[s] % n + g))
            f = m == -1
            if f.any():
                rst_d.append(dst[f])
                rst_s.append(restrict_src(L, X[f], Y[f], Z[f]))
            c = m == -2
            if c.any():
                Xf, Yf, Zf = X[c], Y[c], Z[c]
                Xc, Yc, Zc = Xf // 2, Yf // 2, Zf // 2
                cc = leaf_at(L - 1, Xc, Yc, Zc)
                assert (cc >= 0).all()
                pro_d.append(dst[c])
                pro_c.append(flat(cc, Zc % n + g, Yc % n + g, Xc % n + g))
                pro_sg.append(np.stack([np.where(Xf % 2 == 1, 1.0, -1.0),
                                        np.where(Yf % 2 == 1, 1.0, -1.0),
                                        np.where(Zf % 2 == 1, 1.0, -1.0)], -1))
                nbi, nbm = [], []
                for ax in range(3):
                    for sgn in (-1, 1):
                        P = [Xc, Yc, Zc]
                        P[ax] = _bc(mesh, L - 1, ax, P[ax] + sgn)
                        i8, md = value0(L - 1, *P)
                        nbi.append(i8)
                        nbm.append(md)
                pro_nb.append(np.stack(nbi, 1))
                pro_mode.append(np.stack(nbm, 1))

        cat = lambda xs, shape: (torch.from_numpy(np.concatenate(xs)) if xs
                                 else torch.zeros(shape, dtype=torch.int64))
        self.copy_d, self.copy_s = cat(copy_d, (0,)), cat(copy_s, (0,))
        self.rst_d, self.rst_s = cat(rst_d, (0,)), cat(rst_s, (0, 8))
        self.pro_d, self.pro_c = cat(pro_d, (0,)), cat(pro_c, (0,))
        self.pro_sg = (torch.from_numpy(np.concatenate(pro_sg)) if pro_sg
                       else torch.zeros((0, 3), dtype=torch.float64))
        self.pro_nb, self.pro_mode = cat(pro_nb, (0, 6, 8)), cat(pro_mode, (0, 6))

    def leaves_read(self):
        """Sorted indices of the leaves the plan reads or writes."""
        per = self.nf * self.N3
        ids = [t.reshape(-1) // per for t in (self.copy_d, self.copy_s, self.rst_d, self.rst_s, self.pro_d,
                                              self.pro_c, self.pro_nb) if t.numel()]
        return np.unique(torch.cat(ids).numpy()) if ids else np.zeros(0, dtype=np.int64)

    def compact(self, leaves):
        """The same plan over a pool that holds only `leaves` (sorted, a
        superset of leaves_read()), leaf leaves[k] at slot k."""
        per = self.nf * self.N3
        pos = torch.full((int(max(leaves)) + 1,), -1, dtype=torch.int64)
        pos[torch.as_tensor(leaves, dtype=torch.int64)] = torch.arange(len(leaves), dtype=torch.int64)
        out = RefreshPlan.__new__(RefreshPlan)
        out.__dict__.update(self.__dict__)
        for name in ("copy_d", "copy_s", "rst_d", "rst_s", "pro_d", "pro_c", "pro_nb"):
            t = getattr(self, name)
            if t.numel():
                slot = pos[t // per]
                assert bool((slot >= 0).all()), "a leaf the plan reads is missing from the pool"
                t = slot * per + t % per
            setattr(out, name, t)
        return out

    def apply(self, U):
        shape = U.shape
        Uf = U.reshape(-1)
        out = Uf.clone()
        fo = (torch.arange(self.nf, dtype=torch.int64) * self.N3).view(self.nf, 1)

        def gather(idx):            # idx [k] -> [nf, k]
            return Uf[idx.view(1, -1) + fo]

        def restrict(idx8):         # idx8 [k, 8] -> [nf, k]
            v = gather(idx8[:, 0])
            for t in range(1, 8):
                v = v + gather(idx8[:, t])
            return v * 0.125

        if self.copy_d.numel():
            out[self.copy_d.view(1, -1) + fo] = gather(self.copy_s)
        if self.rst_d.numel():
            out[self.rst_d.view(1, -1) + fo] = restrict(self.rst_s)
        if self.pro_d.numel():
            Uc = gather(self.pro_c)
            nb = []
            for e in range(6):
                single = gather(self.pro_nb[:, e, 0])
                mean = restrict(self.pro_nb[:, e, :])
                nb.append(torch.where(self.pro_mode[:, e].view(1, -1) == 1, mean, single))
            D = [minmod(Uc - nb[2 * ax], nb[2 * ax + 1] - Uc) for ax in range(3)]
            sg = self.pro_sg.t().unsqueeze(1)       # [3, 1, k]
            Uf_new = Uc + 0.25 * ((sg[0] * D[0] + sg[1] * D[1]) + sg[2] * D[2])
            out[self.pro_d.view(1, -1) + fo] = Uf_new
        return out.view(shape)


def minmod(a, b):
    return torch.where(a * b > 0.0, torch.where(torch.abs(a) <= torch.abs(b), a, b), torch.zeros_like(a))


def ghost_refresh(U, mesh: Mesh, plan: RefreshPlan | None = None):
    return (plan or RefreshPlan(mesh)).apply(U)


# ---------------------------------------------------------- flux correction
FACE_ORDER = [(0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)]


def coarse_fine_faces(mesh: Mesh):
    """(coarse leaf, axis, side, [(fine leaf, o1, o2) x4]) for every face of a
    leaf whose same-level neighbour node is refined; o1, o2 are the child
    octant bits along the two transverse axes (t1 < t2)."""
    maps = mesh.maps()
    out = []
    for b, (L, i, j, k) in enumerate(mesh.leaves):
        L, i, j, k = int(L), int(i), int(j), int(k)
        for axis, side in FACE_ORDER:
            off = [0, 0, 0]
            off[axis] = side
            ni, nj, nk = (mesh.wrap(L, 0, i + off[0]), mesh.wrap(L, 1, j + off[1]),
                          mesh.wrap(L, 2, k + off[2]))
            if ni is None or nj is None or nk is None or maps[L][nk, nj, ni] != -1:
                continue
            t = [a for a in range(3) if a != axis]
            kids = []
            for o1 in (0, 1):
                for o2 in (0, 1):
                    o = [0, 0, 0]
                    o[axis] = 1 if side < 0 else 0
                    o[t[0]], o[t[1]] = o1, o2
                    f = int(maps[L + 1][2 * nk + o[2], 2 * nj + o[1], 2 * ni + o[0]])
                    assert f >= 0
                    kids.append((f, o1, o2))
            out.append((b, axis, side, kids))
    return out


def flux_correct(U, mesh: Mesh, faces, dt: float, cf=None):
    """Replace the coarse flux at every coarse-fine face by the mean of the
    four fine fluxes over it (one global dt, no subcycling):
    U_c += s*(dt/dx_c)*(F_c - 0.25*((F00 + F10) + (F01 + F11))), s = +1 on
    the coarse cell's high face, -1 on its low face, faces in the order
    -x, +x, -y, +y, -z, +z."""
    d = mesh.desc
    n, g = d.n, d.ghosts
    h = n // 2
    cf = coarse_fine_faces(mesh) if cf is None else cf
    if not cf:
        return U
    U = U.clone()
    dxs = dx_of_leaves(mesh)
    for b, axis, side, kids in cf:
        dtdx = dt / float(dxs[b])
        Fc = faces[axis][1 if side > 0 else 0][b]            # [nf, n(t2), n(t1)]
        for f, o1, o2 in kids:
            Ff = faces[axis][0 if side > 0 else 1][f]       # fine leaf, opposite face
            F00 = Ff[:, 0::2, 0::2]
            F10 = Ff[:, 0::2, 1::2]
            F01 = Ff[:, 1::2, 0::2]
            F11 = Ff[:, 1::2, 1::2]
            mean = ((F00 + F10) + (F01 + F11)) * 0.25       # [nf, h(t2), h(t1)]
            sl2 = slice(o2 * h, (o2 + 1) * h)
            sl1 = slice(o1 * h, (o1 + 1) * h)
            corr = (dtdx * (Fc[:, sl2, sl1] - mean)) * float(side)
            cell = g + n - 1 if side > 0 else g
            t1, t2 = [a for a in range(3) if a != axis]
            idx = [slice(None)] * 5
            idx[0] = b
            idx[AXIS_DIM[axis]] = cell
            idx[AXIS_DIM[t1]] = slice(g + o1 * h, g + (o1 + 1) * h)
            idx[AXIS_DIM[t2]] = slice(g + o2 * h, g + (o2 + 1) * h)
            U[tuple(idx)] = U[tuple(idx)] + corr
    return U


# ------------------------------------------------------ reductions and step
def lab_primitives(U, gamma):
    """(rho, u, v, w, p) in lab order; with a sixth field (dual energy) the
    pressure is selected as in primitives."""
    rho = torch.clamp_min(U[:, 0], RHO_FLOOR)
    u, v, w = U[:, 1] / rho, U[:, 2] / rho, U[:, 3] / rho
    ke = (0.5 * rho) * (u * u + (v * v + w * w))
    if U.shape[1] == 5:
        p = torch.clamp_min((gamma - 1.0) * (U[:, 4] - ke), P_FLOOR)
    else:
        eint = U[:, 4] - ke
        p = torch.clamp_min((gamma - 1.0) * torch.where(eint > DE_ETA1 * U[:, 4], eint, U[:, 5]), P_FLOOR)
    return rho, u, v, w, p


def reduce_dt_totals(U, mesh: Mesh, cfl: float):
    """dt = cfl * min over leaf interior cells of dx_L / (max(|u|,|v|,|w|) + c),
    c = sqrt(gamma*p/rho); totals = sum over leaves of dx_L^3 * sum of U over
    the five conserved fields (rho e of the dual-energy formalism is not a
    conserved quantity and has no total)."""
    d = mesh.desc
    n, g = d.n, d.ghosts
    I = U[:, :, g:g + n, g:g + n, g:g + n]
    rho, u, v, w, p = lab_primitives(I, d.gamma)
    c = ieee_sqrt((d.gamma * p) / rho)
    s = torch.maximum(torch.abs(u), torch.maximum(torch.abs(v), torch.abs(w))) + c
    dx = dx_of_leaves(mesh).view(-1, 1, 1, 1)
    dt = cfl * float(torch.min(dx / s))
    vol = dx.view(-1) ** 3
    totals = (I[:, :5].sum(dim=(2, 3, 4)) * vol.view(-1, 1)).sum(0)
    return dt, totals


def step(U, mesh: Mesh, dt: float, cycle: int, plan: RefreshPlan | None = None,
         flux_correction: bool = True, cf=None):
    """One hydro step: ghost refresh, three split PPM sweeps, coarse-fine flux
    correction.  dt is given (the caller takes it from reduce_dt_totals or
    from a fixed sequence)."""
    U = ghost_refresh(U, mesh, plan)
    faces = {}
    swept = set()
    for axis in sweep_order(cycle):
        U, faces[axis] = sweep(U, mesh, axis, dt, transverse_rows(mesh, axis, swept))
        swept.add(axis)
    if flux_correction:
        U = flux_correct(U, mesh, faces, dt, cf)
    return U


def run(U, mesh: Mesh, steps: int, cfl: float, dts=None, cycle0: int = 0):
    """Advance `steps` steps; dt from the CFL reduction of the state at the
    start of each step unless a fixed sequence dts is given.  Returns
    (U, list of dt used)."""
    plan = RefreshPlan(mesh)
    cf = coarse_fine_faces(mesh)
    used = []
    for s in range(steps):
        dt = float(dts[s]) if dts is not None else reduce_dt_totals(U, mesh, cfl)[0]
        U = step(U, mesh, dt, cycle0 + s, plan, cf=cf)
        used.append(dt)
    return U, used


# ------------------------------------------------------------ refine flags
def refine_flags(U, mesh: Mesh, field: int, tau: float, tau_c: float):
    """Per-leaf flag from the relative-slope criterion on density (field 0) or
    pressure (field 4), compared in float64 on cells of the (ghost-refreshed)
    leaf interior: a cell passes on axis d if |q(i+e_d) - q(i-e_d)| >
    (2*tau)*|q(i)|.  +1 if any cell passes and L < max_level; -1 if none
    passes with tau_c and L > 0; 0 otherwise."""
    d = mesh.desc
    n, g = d.n, d.ghosts
    Ud = U.to(torch.float64)
    if field == 0:
        q = torch.clamp_min(Ud[:, 0], RHO_FLOOR)
    else:
        q = lab_primitives(Ud, d.gamma)[4]
    thr, thr_c = 2.0 * tau, 2.0 * tau_c
    c = q[:, g:g + n, g:g + n, g:g + n]
    hit = torch.zeros(U.shape[0], dtype=torch.bool)
    hit_c = torch.zeros(U.shape[0], dtype=torch.bool)
    for axis in range(3):
        lo = [slice(None), slice(g, g + n), slice(g, g + n), slice(g, g + n)]
        hi = list(lo)
        dim = 3 - axis
        lo[dim] = slice(g - 1, g + n - 1)
        hi[dim] = slice(g + 1, g + n + 1)
        diff = torch.abs(q[tuple(hi)] - q[tuple(lo)])
        hit |= (diff > thr * torch.abs(c)).flatten(1).any(1)
        hit_c |= (diff > thr_c * torch.abs(c)).flatten(1).any(1)
    L = torch.from_numpy(mesh.leaves[:, 0])
    flags = torch.zeros(U.shape[0], dtype=torch.int8)
    flags[(~hit_c) & (L > 0)] = -1
    flags[hit & (L < d.max_level)] = 1
    return flags


# ------------------------------------------------------------------- remap
def remap(U_old, old: Mesh, new: Mesh):
    """Field data of a rebuilt mesh (Sec. II.B: Refine with Prolong and
    Restrict move data between levels).  U_old must have refreshed ghosts.
    Per new leaf, interior cells only (ghosts are left zero):
      * the same leaf existed: copy;
      * an old leaf k levels coarser contains it: conservative minmod-limited
        linear reconstruction of the old cell C evaluated at the new cell
        centre, U = U_C + ((xi_x D_x + xi_y D_y) + xi_z D_z), xi the centre
        offset in units of the old cell width (+-1/4 for k = 1; +-1/8, +-3/8
        for k = 2), D_d = minmod(U_C - U_C-e_d, U_C+e_d - U_C) from the old
        leaf's padded block;
      * its 8 children were old leaves: restriction, mean of the 8 old cells
        in (dz, dy, dx) order times 0.125."""
    d = new.desc
    n, g = d.n, d.ghosts
    N = n + 2 * g
    out = torch.zeros((new.n_leaves, U_old.shape[1], N, N, N), dtype=U_old.dtype)
    r = torch.arange(n)
    for b, (L, i, j, k) in enumerate(new.leaves):
        L, i, j, k = int(L), int(i), int(j), int(k)
        t = (L, i, j, k)
        if t in old.index:
            src = old.index[t]
            out[b, :, g:g + n, g:g + n, g:g + n] = U_old[src, :, g:g + n, g:g + n, g:g + n]
            continue
        anc = None
        for kk in range(1, L + 1):
            a = (L - kk, i >> kk, j >> kk, k >> kk)
            if a in old.index:
                anc = (old.index[a], kk, a)
                break
        if anc is not None:
            src, kk, a = anc
            A = U_old[src]
            cell = [((c0 * n + r) >> kk) - a[1 + ax] * n + g for ax, c0 in enumerate((i, j, k))]
            xi = [(((c0 * n + r) % (1 << kk)).to(torch.float64) + 0.5) / (1 << kk) - 0.5 for c0 in (i, j, k)]
            cz, cy, cx = cell[2].view(-1, 1, 1), cell[1].view(1, -1, 1), cell[0].view(1, 1, -1)
            Uc = A[:, cz, cy, cx]
            D = []
            for ax, (oz, oy, ox) in enumerate(((0, 0, 1), (0, 1, 0), (1, 0, 0))):
                Um = A[:, cz - oz, cy - oy, cx - ox]
                Up = A[:, cz + oz, cy + oy, cx + ox]
                D.append(minmod(Uc - Um, Up - Uc))
            xz, xy, xx = xi[2].view(1, -1, 1, 1), xi[1].view(1, 1, -1, 1), xi[0].view(1, 1, 1, -1)
            out[b, :, g:g + n, g:g + n, g:g + n] = Uc + ((xx * D[0] + xy * D[1]) + xz * D[2])
            continue
        h = n // 2
        for o in range(8):
            ox, oy, oz = o & 1, (o >> 1) & 1, o >> 2
            c = (L + 1, 2 * i + ox, 2 * j + oy, 2 * k + oz)
            assert c in old.index, "meshes are not one adaptation apart"
            C = U_old[old.index[c]]
            v = None
            for dz in (0, 1):
                for dy in (0, 1):
                    for dx in (0, 1):
                        blk = C[:, g + dz:g + n:2, g + dy:g + n:2, g + dx:g + n:2]
                        v = blk if v is None else v + blk
            out[b, :, g + oz * h:g + (oz + 1) * h, g + oy * h:g + (oy + 1) * h, g + ox * h:g + (ox + 1) * h] = v * 0.125
    return out


def adapt(U, mesh: Mesh, field: int = 0, tau: float = 0.3, tau_c: float | None = None):
    """Refresh, flag, rebuild and remap (the oracle's adaptation step)."""
    from .mesh import build
    tau_c = tau / 4 if tau_c is None else tau_c
    U = ghost_refresh(U, mesh)
    flags = refine_flags(U, mesh, field, tau, tau_c).numpy()
    if not flags.any():
        return mesh, U, flags
    new = build(mesh.desc, mesh, flags)
    if np.array_equal(new.leaves, mesh.leaves):
        return mesh, U, flags
    return new, remap(U, mesh, new), flags
