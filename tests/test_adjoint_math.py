"""CPU checks of the per-interface PPM arithmetic of the CUDA path and of its
hand-written adjoint (compiled for the host from the same device functions):
the flux equals the oracle's bit for bit in float64, and the adjoint equals
torch autograd through the oracle (Sec. II.C PPM, dt held fixed)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import hydro as OH


@pytest.fixture(scope="module")
def hc():
    from paper_1810_01319_gb300 import build
    L = ctypes.CDLL(build.build_hostcheck())
    dp = ctypes.POINTER(ctypes.c_double)
    L.cello_hc_window_flux.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
    L.cello_hc_window_flux_vjp.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp]
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _windows(seed, count):
    """8-cell windows of conserved states: smooth data, jumps (shocks,
    contacts, rarefactions), moving and at rest."""
    rng = np.random.default_rng(seed)
    out = []
    for w in range(count):
        x = np.arange(8)
        kind = w % 4
        rho = 1.0 + 0.3 * rng.standard_normal(8) * (kind == 0)
        p = 1.0 + 0.3 * rng.standard_normal(8) * (kind == 0)
        if kind >= 1:
            cut = rng.integers(2, 6)
            rho = np.where(x < cut, rng.uniform(0.5, 3), rng.uniform(0.1, 1.0))
            p = np.where(x < cut, rng.uniform(1, 10), rng.uniform(0.05, 1.0))
            rho *= 1 + 0.05 * rng.random(8)
            p *= 1 + 0.05 * rng.random(8)
        u = rng.uniform(-1.5, 1.5) + 0.3 * rng.standard_normal(8)
        if kind == 2:
            u = np.where(x < 4, 1.5, -1.5) + 0.1 * rng.random(8)   # colliding: strong shock
        v = 0.2 * rng.standard_normal(8)
        wv = 0.2 * rng.standard_normal(8)
        rho = np.abs(rho) + 0.05
        p = np.abs(p) + 0.05
        gamma = 1.4
        E = p / (gamma - 1) + 0.5 * rho * (u * u + v * v + wv * wv)
        out.append(np.stack([rho, rho * u, rho * v, rho * wv, E], 1))
    return out


def _oracle_flux(U8, dtdx, gamma):
    Uc = [U8[:, k] for k in range(5)]
    F = OH.pencil_fluxes(Uc, dtdx, gamma)
    return torch.stack([f[..., 0] for f in F])


def test_window_flux_bit_exact_with_oracle(hc):
    for U in _windows(0, 200):
        dtdx = 0.3
        F = np.zeros(5)
        hc.cello_hc_window_flux(_ptr(np.ascontiguousarray(U)), dtdx, 1.4, 8, _ptr(F))
        Fo = _oracle_flux(torch.from_numpy(U), dtdx, 1.4).numpy()
        assert np.array_equal(F, Fo), (F, Fo)


def test_window_flux_adjoint_matches_autograd(hc):
    rng = np.random.default_rng(1)
    worst = 0.0
    for U in _windows(2, 200):
        dtdx = 0.3
        Fb = rng.standard_normal(5)
        Ub = np.zeros((8, 5))
        hc.cello_hc_window_flux_vjp(_ptr(np.ascontiguousarray(U)), dtdx, 1.4, 8, _ptr(Fb), _ptr(Ub))
        Ut = torch.from_numpy(U.copy()).requires_grad_(True)
        F = _oracle_flux(Ut, dtdx, 1.4)
        (g,) = torch.autograd.grad(F, Ut, torch.from_numpy(Fb))
        g = g.numpy()
        scale = np.abs(g).max() + 1e-300
        worst = max(worst, np.abs(Ub - g).max() / scale)
    assert worst < 1e-11, worst


def test_window_flux_adjoint_float32_close(hc):
    rng = np.random.default_rng(3)
    for U in _windows(4, 40):
        Fb = rng.standard_normal(5)
        U64 = np.zeros((8, 5))
        U32 = np.zeros((8, 5))
        c = np.ascontiguousarray(U)
        hc.cello_hc_window_flux_vjp(_ptr(c), 0.3, 1.4, 8, _ptr(Fb), _ptr(U64))
        hc.cello_hc_window_flux_vjp(_ptr(c), 0.3, 1.4, 4, _ptr(Fb), _ptr(U32))
        assert np.abs(U32 - U64).max() <= 1e-3 * (np.abs(U64).max() + 1e-30)
