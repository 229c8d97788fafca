"""Reference solutions used to pin the oracle.  TEST INFRASTRUCTURE ONLY.

* Exact Riemann solver for the ideal-gas Euler equations (the textbook
  construction: pressure function with shock and rarefaction branches, Newton
  iteration on p*, self-similar sampling).  It pins the Sod runs and the
  two-shock approximate solver of the method.
* Sedov-Taylor point blast: the similarity constant xi0 of R = xi0 *
  (E t^2 / rho0)^(1/5), obtained by integrating the self-similar ODEs behind
  the strong shock and evaluating the energy integral.
"""
from __future__ import annotations

import math

import numpy as np


# ------------------------------------------------------------ exact Riemann
def _pressure_fn(p, rho, pk, c, gamma):
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        Bc = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + Bc))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (Bc + p))
    e = (gamma - 1.0) / (2.0 * gamma)
    return (2.0 * c / (gamma - 1.0)) * ((p / pk) ** e - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * c)


def star_state(rL, uL, pL, rR, uR, pR, gamma, tol=1e-15):
    """(p*, u*) of the exact Riemann problem, Newton to relative tol."""
    cL, cR = math.sqrt(gamma * pL / rL), math.sqrt(gamma * pR / rR)
    p = max(1e-12, 0.5 * (pL + pR) - 0.125 * (uR - uL) * (rL + rR) * (cL + cR))
    for _ in range(200):
        fL, dL = _pressure_fn(p, rL, pL, cL, gamma)
        fR, dR = _pressure_fn(p, rR, pR, cR, gamma)
        pn = p - (fL + fR + uR - uL) / (dL + dR)
        pn = max(pn, 1e-14 * p)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _pressure_fn(p, rL, pL, cL, gamma)
    fR, _ = _pressure_fn(p, rR, pR, cR, gamma)
    return p, 0.5 * (uL + uR) + 0.5 * (fR - fL)


def sample(xi, rL, uL, pL, rR, uR, pR, gamma):
    """Exact (rho, u, p) at similarity coordinate xi = x/t (arrays allowed)."""
    ps, us = star_state(rL, uL, pL, rR, uR, pR, gamma)
    xi = np.asarray(xi, dtype=np.float64)
    g = gamma
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    out = np.empty(xi.shape + (3,))
    for idx, s in np.ndenumerate(xi):
        if s <= us:                                     # left of the contact
            if ps > pL:
                rs = rL * ((ps / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pL + 1))
                S = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                out[idx] = (rL, uL, pL) if s <= S else (rs, us, ps)
            else:
                rs = rL * (ps / pL) ** (1 / g)
                cs = cL * (ps / pL) ** ((g - 1) / (2 * g))
                if s <= uL - cL:
                    out[idx] = (rL, uL, pL)
                elif s >= us - cs:
                    out[idx] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    r = rL * (c / cL) ** (2 / (g - 1))
                    out[idx] = (r, u, pL * (c / cL) ** (2 * g / (g - 1)))
        else:
            if ps > pR:
                rs = rR * ((ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1))
                S = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                out[idx] = (rR, uR, pR) if s >= S else (rs, us, ps)
            else:
                rs = rR * (ps / pR) ** (1 / g)
                cs = cR * (ps / pR) ** ((g - 1) / (2 * g))
                if s >= uR + cR:
                    out[idx] = (rR, uR, pR)
                elif s <= us + cs:
                    out[idx] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    r = rR * (c / cR) ** (2 / (g - 1))
                    out[idx] = (r, u, pR * (c / cR) ** (2 * g / (g - 1)))
    return out[..., 0], out[..., 1], out[..., 2]


# ------------------------------------------------------------- Sedov-Taylor
def sedov_xi0(gamma: float, nu: int = 3, npts: int = 20000) -> float:
    """Similarity constant of the strong point blast in nu dimensions.

    Behind the shock R(t) = xi0 (E t^2/rho0)^(1/(nu+2)) the flow is
    self-similar in lam = r/R: rho = rho0*G(lam), u = Rdot*V(lam),
    p = rho0*Rdot^2*P(lam).  With a = 2/(nu+2) (R ~ t^a) the mass, momentum
    and entropy equations become three ODEs in lam, integrated inward from
    the strong-shock values G = (g+1)/(g-1), V = 2/(g+1), P = 2/(g+1) at
    lam = 1.  Energy: E = xi0^(nu+2) * rho0 * a^2 * S_nu * integral of
    (G V^2/2 + P/(g-1)) lam^(nu-1) dlam, S_3 = 4 pi, S_2 = 2 pi, S_1 = 2."""
    g = gamma
    a = 2.0 / (nu + 2)

    # Unknowns y = (G, V, P) as functions of lam; with f' = d/dlam.
    # continuity:  -lam G' + (G V)' + (nu-1) G V / lam = 0
    # momentum:    G (V - lam) V' + P' = -(1 - 1/a) G V          [Rddot R / Rdot^2 = 1 - 1/a]
    # entropy:     (V - lam) (P'/P - g G'/G) = -2 (1 - 1/a), from d/dt ln(p rho^-g) = 0
    #   along particle paths with p/rho^g ~ Rdot^2 P / G^g.
    k = 1.0 - 1.0 / a

    def rhs(lam, y):
        G, V, P = y
        w = V - lam
        # linear system M y' = b
        M = np.array([[w, G, 0.0],
                      [0.0, G * w, 1.0],
                      [-g * w / G, 0.0, w / P]])
        b = np.array([-(nu - 1) * G * V / lam,
                      -k * G * V,
                      -2.0 * k])
        return np.linalg.solve(M, b)

    lam = 1.0
    y = np.array([(g + 1) / (g - 1), 2.0 / (g + 1), 2.0 / (g + 1)])
    lam_end = 1e-4
    h = -(1.0 - lam_end) / npts
    integ = 0.0

    def integrand(lam, y):
        G, V, P = y
        return (0.5 * G * V * V + P / (g - 1.0)) * lam ** (nu - 1)

    f_prev = integrand(lam, y)
    for _ in range(npts):
        k1 = rhs(lam, y)
        k2 = rhs(lam + 0.5 * h, y + 0.5 * h * k1)
        k3 = rhs(lam + 0.5 * h, y + 0.5 * h * k2)
        k4 = rhs(lam + h, y + h * k3)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        lam = lam + h
        f_new = integrand(lam, y)
        integ += -h * 0.5 * (f_prev + f_new)
        f_prev = f_new
    S = {1: 2.0, 2: 2.0 * math.pi, 3: 4.0 * math.pi}[nu]
    alpha = a * a * S * integ
    return alpha ** (-1.0 / (nu + 2))
