"""GPU adjoint of the hydro step (dt fixed) against torch autograd through
the float64 oracle, against central finite differences of the GPU forward,
and float32 against float64."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM

pytestmark = pytest.mark.gpu


def _periodic(root=(2, 2, 2), n=8):
    od = OM.Desc(root=root, n=n, ghosts=4, max_level=0, bc=(OM.PERIODIC,) * 3, gamma=5.0 / 3.0,
                 hi=tuple(r / max(root) for r in root))
    return od, OM.root_mesh(od)


def _moving_state(od, om, seed):
    U = H.state(od, om.leaves, "blobs", count=6, seed=seed)
    g = torch.Generator().manual_seed(seed)
    U[:, 0] *= 1.0 + 0.2 * torch.rand(U[:, 0].shape, generator=g, dtype=torch.float64)
    U[:, 4] *= 1.0 + 0.5 * torch.rand(U[:, 4].shape, generator=g, dtype=torch.float64)
    return U


@pytest.mark.parametrize("steps,n", [(1, 8), (2, 8), (3, 16)])
def test_adjoint_matches_oracle_autograd(steps, n):
    od, om = _periodic(n=n)
    U0 = _moving_state(od, om, 3)
    _, dts = OH.run(U0, om, steps, 0.4)
    w = torch.randn(U0.shape, generator=torch.Generator().manual_seed(7), dtype=torch.float64)
    g4 = od.ghosts
    wi = torch.zeros_like(w)
    wi[:, :, g4:g4 + n, g4:g4 + n, g4:g4 + n] = w[:, :, g4:g4 + n, g4:g4 + n, g4:g4 + n]
    # oracle gradient of sum(w * U_final) by autograd
    Ut = U0.clone().requires_grad_(True)
    plan = OH.RefreshPlan(om)
    V = Ut
    for s, dt in enumerate(dts):
        V = OH.step(V, om, dt, s, plan)
    (go,) = torch.autograd.grad((V * wi).sum(), Ut)
    # GPU adjoint
    gm = H.gpu_mesh_from_flags(od, [], 8)
    U = U0.cuda().contiguous()
    states = []
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s, v in enumerate(dts):
        states.append(U.clone())
        dt.fill_(v)
        gm.hydro_step(U, dt, s)
    lam = wi.cuda().contiguous()
    for s in range(steps - 1, -1, -1):
        dt.fill_(dts[s])
        gm.hydro_adjoint_step(states[s], lam, dt, s)
    torch.cuda.synchronize()
    gg = lam.cpu()
    err = float((gg - go).abs().max() / go.abs().max())
    assert err < 1e-10, err


def _loss(gm, rho0, base, dts, target, every=5):
    from paper_1810_01319_gb300.autograd import rollout
    U0 = base.clone()
    U0[:, 0] = rho0
    U0[:, 4] = base[:, 4]                 # p = 1, v = 0: E does not depend on rho
    Uf = rollout(gm, U0, dts, 0, every)
    g = 4
    n = gm.desc.n
    rho = Uf[:, 0, g:g + n, g:g + n, g:g + n]
    return ((rho - target) ** 2).sum()


@pytest.mark.parametrize("root,n,steps,ndir", [((2, 2, 2), 16, 20, 6), ((4, 4, 4), 32, 50, 16)])
def test_gradient_against_finite_differences(root, n, steps, ndir):
    """Adjoint workload: rho0 = 1 + 0.1 GRF(k^-2, seed 0), p = 1, v = 0,
    gamma 5/3, periodic; loss = sum (rho_final - rho_target)^2 with the
    target from seed 1; gradient wrt rho0 checked on random directions by
    central differences (float64, frozen dt).  The step is 1e-4 of the rms
    density along a unit direction: smaller steps are dominated by the
    rounding noise of 50 nonlinear steps (measured: relative FD error 4e-7 at
    1e-4, 2e-5 at 1e-5, 3e-4 at 1e-6)."""
    od, om = _periodic(root=root, n=n)
    gm = H.gpu_mesh_from_flags(od, [], 8)
    base = H.state(od, om.leaves, "grf", seed=0).cuda()
    tgt0 = H.state(od, om.leaves, "grf", seed=1).cuda()
    dts = []
    U = base.clone().contiguous()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s in range(steps):
        gm.reduce(U, 0.4, dt_next=dt)
        dts.append(float(dt))
        gm.hydro_step(U, dt, s)
    from paper_1810_01319_gb300.autograd import rollout
    Ut = rollout(gm, tgt0.contiguous(), dts, 0, 10)
    target = Ut[:, 0, 4:4 + n, 4:4 + n, 4:4 + n].clone()
    rho0 = base[:, 0].clone().requires_grad_(True)
    L = _loss(gm, rho0, base, dts, target)
    (grad,) = torch.autograd.grad(L, rho0)
    gen = torch.Generator(device="cuda").manual_seed(5)
    worst = 0.0
    for k in range(ndir):
        d = torch.randn(rho0.shape, generator=gen, device="cuda", dtype=torch.float64)
        d[:, :4] = 0; d[:, -4:] = 0; d[:, :, :4] = 0; d[:, :, -4:] = 0; d[:, :, :, :4] = 0; d[:, :, :, -4:] = 0
        d /= d.norm()
        eps = 1e-4 * float(rho0.detach().norm()) / np.sqrt(rho0.numel())
        with torch.no_grad():
            lp = float(_loss(gm, rho0.detach() + eps * d, base, dts, target))
            lm = float(_loss(gm, rho0.detach() - eps * d, base, dts, target))
        fd = (lp - lm) / (2 * eps)
        an = float((grad * d).sum())
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-30))
    assert worst < 1e-4, worst


def test_float32_gradient_against_finite_differences():
    """The adjoint workload (4^3 roots of 32^3 cells = 128^3, 50 steps) on the
    float32 path: the float32 adjoint's directional derivatives against
    central differences of the float32 forward (frozen dt from the float32
    CFL reduction), on 16 directions.

    A step suited to float32: each direction is a smooth field (the same
    k^-2 random-field recipe as the initial density, seeds 100-115, zero in
    the ghosts, unit norm) and eps = 1e-4 sqrt(cells), so the perturbation
    is ~1e-4 per cell (~1700 float32 ulp of the unit density, small next to
    the field's 0.1 amplitude) and the loss is summed in float64.  Budget:
    the float32 rounding noise of the forward enters (L+ - L-) at ~1e-5 of
    the signal, the O(eps^2) truncation at ~1e-6, and the float32 adjoint's
    own rounding (50 reverse steps) at ~1e-4; tolerance 2e-3 relative."""
    root, n, steps, ndir = (4, 4, 4), 32, 50, 16
    od, om = _periodic(root=root, n=n)
    gm = H.gpu_mesh_from_flags(od, [], 4)
    base = H.state(od, om.leaves, "grf", seed=0).to(torch.float32).cuda()
    tgt0 = H.state(od, om.leaves, "grf", seed=1).to(torch.float32).cuda()
    dts = []
    U = base.clone().contiguous()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s in range(steps):
        gm.reduce(U, 0.4, dt_next=dt)
        dts.append(float(dt))
        gm.hydro_step(U, dt, s)
    from paper_1810_01319_gb300.autograd import rollout
    g4 = 4
    target = rollout(gm, tgt0.contiguous(), dts, 0, 10)[:, 0, g4:g4 + n, g4:g4 + n, g4:g4 + n].double()

    def loss(rho0):
        U0 = base.clone()
        U0[:, 0] = rho0
        Uf = rollout(gm, U0, dts, 0, 10)
        return ((Uf[:, 0, g4:g4 + n, g4:g4 + n, g4:g4 + n].double() - target) ** 2).sum()

    rho0 = base[:, 0].clone().requires_grad_(True)
    (grad,) = torch.autograd.grad(loss(rho0), rho0)
    cells = om.n_leaves * n ** 3
    eps = 1e-4 * np.sqrt(cells)
    worst = 0.0
    for k in range(ndir):
        d = H.state(od, om.leaves, "grf", seed=100 + k)[:, 0] - 1.0
        d[:, :g4] = 0; d[:, -g4:] = 0; d[:, :, :g4] = 0; d[:, :, -g4:] = 0; d[:, :, :, :g4] = 0; d[:, :, :, -g4:] = 0
        d = (d / d.norm()).cuda()
        with torch.no_grad():
            rp = rho0.detach() + (eps * d).float()
            rm = rho0.detach() - (eps * d).float()
            lp, lm = float(loss(rp)), float(loss(rm))
        fd = (lp - lm) / (2 * eps)
        # along the perturbation float32 actually applied (rp - rm)
        an = float((grad.double() * (rp.double() - rm.double())).sum()) / (2 * eps)
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-30))
    print(f"float32 adjoint vs central differences, 128^3 x 50 steps: worst relative error {worst:.2e}")
    assert worst < 2e-3, worst


def test_float32_adjoint_close_to_float64():
    od, om = _periodic(n=16)
    U0 = _moving_state(od, om, 9)
    _, dts = OH.run(U0, om, 2, 0.4)
    out = {}
    for prec in (8, 4):
        gm = H.gpu_mesh_from_flags(od, [], prec)
        U = U0.to(gm.dtype).cuda().contiguous()
        states = []
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        for s, v in enumerate(dts):
            states.append(U.clone())
            dt.fill_(v)
            gm.hydro_step(U, dt, s)
        lam = torch.ones_like(U)
        for s in (1, 0):
            dt.fill_(dts[s])
            gm.hydro_adjoint_step(states[s], lam, dt, s)
        out[prec] = lam.double().cpu()
    err = float((out[4] - out[8]).abs().max() / out[8].abs().max())
    assert err < 1e-3, err


@pytest.mark.parametrize("bc,steps", [((OM.PERIODIC,) * 3, 2), ((OM.OUTFLOW, OM.PERIODIC, OM.OUTFLOW), 2)])
def test_amr_adjoint_matches_oracle_autograd(bc, steps):
    """AMR adjoint (restriction, limited prolongation, coarse-fine flux
    correction, outflow clamps transposed) against torch autograd through the
    oracle on a 2^3-root, level-2 blob mesh."""
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=2, bc=bc)
    om, flags = H.ic_refined(od, "blobs", count=16, seed=2)
    assert om.leaves[:, 0].max() == 2 and len(OH.coarse_fine_faces(om)) > 0
    U0 = _moving_state(od, om, 4)
    _, dts = OH.run(U0, om, steps, 0.4)
    n, g4 = od.n, od.ghosts
    w = torch.randn(U0.shape, generator=torch.Generator().manual_seed(8), dtype=torch.float64)
    wi = torch.zeros_like(w)
    wi[:, :, g4:g4 + n, g4:g4 + n, g4:g4 + n] = w[:, :, g4:g4 + n, g4:g4 + n, g4:g4 + n]
    Ut = U0.clone().requires_grad_(True)
    plan = OH.RefreshPlan(om)
    cf = OH.coarse_fine_faces(om)
    V = Ut
    for s, dt in enumerate(dts):
        V = OH.step(V, om, dt, s, plan, cf=cf)
    (go,) = torch.autograd.grad((V * wi).sum(), Ut)
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    U = U0.cuda().contiguous()
    states = []
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s, v in enumerate(dts):
        states.append(U.clone())
        dt.fill_(v)
        gm.hydro_step(U, dt, s)
    lam = wi.cuda().contiguous()
    for s in range(steps - 1, -1, -1):
        dt.fill_(dts[s])
        gm.hydro_adjoint_step(states[s], lam, dt, s)
    torch.cuda.synchronize()
    err = float((lam.cpu() - go).abs().max() / go.abs().max())
    assert err < 1e-10, err
