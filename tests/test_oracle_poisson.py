"""Pins of the oracle's multigrid Poisson solver (Sec. II.C: mg0, a geometric
multigrid V-cycle): the converged solution against the exact solution of
the same discrete equations by FFT (the 7-point operator is diagonal in
Fourier space), second-order convergence on a manufactured solution, a
steady residual reduction per V-cycle, and the restriction / prolongation
identities."""
import math

import numpy as np
import torch

from oracle import mesh as M
from oracle import poisson as P


def _fft_solve(f, h):
    Mn = f.shape[0]
    k = np.fft.fftfreq(Mn) * Mn
    lam1 = (2.0 * np.cos(2.0 * np.pi * k / Mn) - 2.0) / (h * h)
    lam = lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]
    F = np.fft.fftn(f.numpy() - f.numpy().mean())
    lam[0, 0, 0] = 1.0
    Phi = F / lam
    Phi[0, 0, 0] = 0.0
    return torch.from_numpy(np.real(np.fft.ifftn(Phi)))


def _random_f(Mn, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(Mn, Mn, Mn, generator=g, dtype=torch.float64)


def test_vcycles_converge_to_the_discrete_solution():
    for Mn in (16, 24):                    # 24: the coarse tail is a 3^3 grid solved by sweeps
        h = 1.0 / Mn
        f = _random_f(Mn, Mn)
        phi, norms = P.solve(f, h, 20)
        exact = _fft_solve(f, h)
        assert float((phi - exact).abs().max()) < 1e-10 * float(exact.abs().max()), Mn
        rates = [b / a for a, b in zip(norms[:-1], norms[1:]) if a > 1e-11]
        assert max(rates) < 0.35, rates


def test_second_order_on_a_manufactured_solution():
    errs = []
    for Mn in (16, 32):
        h = 1.0 / Mn
        x = (torch.arange(Mn, dtype=torch.float64) + 0.5) * h
        Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
        s = torch.sin(2 * math.pi * X) * torch.sin(2 * math.pi * Y) * torch.sin(2 * math.pi * Z)
        f = -3.0 * (2 * math.pi) ** 2 * s
        phi, _ = P.solve(f, h, 12)
        errs.append(float((phi - s).abs().max()))
    assert errs[1] < errs[0] / 3.5, errs       # ratio -> 4 for a second-order scheme


def test_restriction_and_prolongation_identities():
    g = torch.Generator().manual_seed(3)
    c = torch.randn(4, 4, 4, generator=g, dtype=torch.float64)
    # prolongation then restriction of a coarse field: a symmetric smoothing
    # (weights 9/16, 3/16 twice... per axis 3/4 * 1/2 + ...), exact on constants
    assert torch.allclose(P.restrict(P.prolong(torch.full((4, 4, 4), 2.5, dtype=torch.float64))),
                          torch.full((4, 4, 4), 2.5, dtype=torch.float64), rtol=0, atol=1e-15)
    # restriction preserves the mean exactly in exact arithmetic
    f = torch.randn(8, 8, 8, generator=g, dtype=torch.float64)
    assert abs(float(P.restrict(f).mean()) - float(f.mean())) < 1e-15
    # prolongation is exact on linear fields away from the periodic seam
    x = torch.arange(4, dtype=torch.float64)
    lin = x.view(1, 1, 4) + 2 * x.view(1, 4, 1) - x.view(4, 1, 1)
    fine = P.prolong(lin)
    xf = (torch.arange(8, dtype=torch.float64) - 0.5) / 2     # fine centres in coarse-cell units
    exact = xf.view(1, 1, 8) + 2 * xf.view(1, 8, 1) - xf.view(8, 1, 1)
    inner = (slice(1, 7),) * 3
    assert torch.allclose(fine[inner], exact[inner], rtol=0, atol=1e-14)


def test_global_grid_round_trip_on_a_uniform_mesh():
    d = M.Desc(root=(2, 2, 2), n=8, ghosts=4, max_level=1)
    mesh = M.build(d, M.root_mesh(d), np.ones(8, dtype=np.int8))
    V = torch.randn(mesh.n_leaves, 8, 8, 8, dtype=torch.float64)
    G = P.to_global(mesh, V)
    assert G.shape == (32, 32, 32) and torch.equal(P.from_global(mesh, G), V)


def test_mixed_precision_cycles_reach_the_float64_solution():
    """float32 V-cycles on the float64 defect: same convergence factor and the
    same discrete solution as the float64 cycles, to 1e-10."""
    for Mn in (16, 24):
        h = 1.0 / Mn
        f = _random_f(Mn, Mn + 1)
        phi, norms = P.solve(f, h, 20, inner="float32")
        exact = _fft_solve(f, h)
        assert float((phi - exact).abs().max()) < 1e-10 * float(exact.abs().max()), Mn
        rates = [b / a for a, b in zip(norms[:6], norms[1:7])]
        assert max(rates) < 0.35, rates
