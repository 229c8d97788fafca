"""GPU hydro step (refresh + PPM sweeps + flux correction + CFL/totals)
against the oracle: float64 within 1e-12 max relative per cell, float32
within 2e-5 L1 relative per field, on the same dt sequence."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM

pytestmark = pytest.mark.gpu


def _run_gpu(gm, U0, steps, dts=None, cfl=0.4, cycle0=0):
    U = U0.to(gm.dtype).cuda().contiguous()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_next = torch.zeros(1, dtype=torch.float64, device="cuda")
    totals = torch.zeros(5, dtype=torch.float64, device="cuda")
    used = []
    if dts is None:
        gm.reduce(U, cfl, dt_next=dt)
    for s in range(steps):
        if dts is not None:
            dt.fill_(float(dts[s]))
        used.append(float(dt.item()))
        gm.hydro_step(U, dt, cycle0 + s, cfl, dt_next=dt_next, totals=totals)
        if dts is None:
            dt.copy_(dt_next)
    torch.cuda.synchronize()
    return U, used, totals.cpu()


@pytest.fixture(scope="module")
def sod_c0():
    """4^3 root blocks of 16^3 cells, Sod along x, outflow x, periodic y/z,
    gamma 1.4, 20 steps at CFL 0.4 (oracle reference)."""
    od = OM.Desc(root=(4, 4, 4), n=16, ghosts=4, max_level=0, bc=(OM.OUTFLOW, OM.PERIODIC, OM.PERIODIC), gamma=1.4)
    om = OM.root_mesh(od)
    U0 = H.state(od, om.leaves, "sod")
    Uo, dts = OH.run(U0, om, 20, 0.4)
    return od, om, U0, Uo, dts


def test_sod_fp64_matches_oracle(sod_c0):
    od, om, U0, Uo, dts = sod_c0
    gm = H.gpu_mesh_from_flags(od, [], 8)
    U, used, _ = _run_gpu(gm, U0, 20)          # the GPU's own CFL dt sequence
    assert np.allclose(used, dts, rtol=1e-12, atol=0)
    err = H.rel_err(H.interior(U, 16), H.interior(Uo, 16))
    assert err <= 1e-12, err


def test_sod_fp32_l1_against_oracle(sod_c0):
    od, om, U0, Uo, dts = sod_c0
    gm = H.gpu_mesh_from_flags(od, [], 4)
    U, _, _ = _run_gpu(gm, U0, 20, dts=dts)
    l1 = H.l1_rel_per_field(H.interior(U, 16), H.interior(Uo, 16))
    assert max(l1) <= 2e-5, l1


@pytest.fixture(scope="module")
def blob_amr():
    """Reduced blob workload: 2^3 root blocks of 16^3 cells, max level 2,
    refined on the density slope of 24 seeded blobs, periodic, gamma 5/3."""
    od = H.oracle_desc(root=(2, 2, 2), n=16, lmax=2)
    om, flags = H.ic_refined(od, "blobs", count=24, seed=0)
    U0 = H.state(od, om.leaves, "blobs", count=24, seed=0)
    Uo, dts = OH.run(U0, om, 6, 0.4)
    assert om.leaves[:, 0].max() == 2 and len(OH.coarse_fine_faces(om)) > 0
    return od, om, flags, U0, Uo, dts


def test_blob_amr_fp64_matches_oracle(blob_amr):
    od, om, flags, U0, Uo, dts = blob_amr
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    assert gm.n_coarse_fine > 0
    U, used, _ = _run_gpu(gm, U0, 6)
    assert np.allclose(used, dts, rtol=1e-12, atol=0)
    err = H.rel_err(H.interior(U, 16), H.interior(Uo, 16))
    assert err <= 1e-12, err


def test_blob_amr_fp32_l1(blob_amr):
    od, om, flags, U0, Uo, dts = blob_amr
    gm = H.gpu_mesh_from_flags(od, flags, 4)
    U, _, _ = _run_gpu(gm, U0, 6, dts=dts)
    l1 = H.l1_rel_per_field(H.interior(U, 16), H.interior(Uo, 16))
    assert max(l1) <= 2e-5, l1


@pytest.mark.parametrize("precision,tol", [(8, 1e-13), (4, 1e-6)])
def test_conservation_on_gpu(blob_amr, precision, tol):
    od, om, flags, U0, Uo, dts = blob_amr
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    U = U0.to(gm.dtype).cuda().contiguous()
    t0 = torch.zeros(5, dtype=torch.float64, device="cuda")
    gm.reduce(U, 0.4, totals=t0)
    Uabs = U.abs()
    scale = torch.zeros(5, dtype=torch.float64, device="cuda")
    gm.reduce(Uabs, 0.4, totals=scale)
    _, _, t1 = _run_gpu(gm, U0, 6, dts=dts)
    drift = ((t1 - t0.cpu()).abs() / scale.cpu())
    assert float(drift.max()) < tol, drift


def test_totals_and_dt_match_oracle(blob_amr):
    od, om, flags, U0, Uo, dts = blob_amr
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    U = U0.cuda().contiguous()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    tot = torch.zeros(5, dtype=torch.float64, device="cuda")
    gm.reduce(U, 0.4, dt_next=dt, totals=tot)
    dto, toto = OH.reduce_dt_totals(U0, om, 0.4)
    assert float(dt) == pytest.approx(dto, rel=1e-15)
    scale = OH.reduce_dt_totals(U0.abs(), om, 0.4)[1]
    assert float(((tot.cpu() - toto).abs() / scale).max()) < 1e-14


@pytest.mark.parametrize("precision", [4, 8])
def test_exec_modes_bit_identical(blob_amr, precision):
    from paper_1810_01319_gb300 import EXEC_BATCHED, EXEC_GRAPH, EXEC_PLAIN
    od, om, flags, U0, Uo, dts = blob_amr
    outs = []
    for mode in (EXEC_PLAIN, EXEC_BATCHED, EXEC_GRAPH):
        gm = H.gpu_mesh_from_flags(od, flags, precision)
        gm.set_exec(mode)
        U, _, tot = _run_gpu(gm, U0, 4)
        outs.append((U.cpu(), tot))
    for U, tot in outs[1:]:
        assert torch.equal(U, outs[0][0]) and torch.equal(tot, outs[0][1])


# float32 sweep variants by form: shared-memory phases, register streaming
F32_SMEM = [0, 1, 2, 3, 4, 5, 12, 13, 14, 15, 16, 17]
F32_STREAM = [6, 7, 8, 9, 10, 11, 18, 19, 20, 21, 22, 23]


@pytest.mark.parametrize("precision", [4, 8])
def test_sweep_variants_identical_and_autotune(blob_amr, precision):
    """Within each form of the sweep (shared-memory phases; register
    streaming), every launch variant (tile shape, register bound, persistent
    schedule) computes the same values.  The two float32 forms evaluate the
    same explicitly rounded expressions (every multiply-add fused or not as
    written, none left to the compiler), so they agree bit for bit too.  The
    autotuner leaves the state unchanged and picks one variant per axis."""
    od, om, flags, U0, Uo, dts = blob_amr
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    forms = [F32_SMEM, F32_STREAM] if precision == 4 else [[0, 1]]
    nv = sum(len(f) for f in forms)
    outs = {}
    for v in range(nv):
        gm.set_sweep_variant(v)
        U, _, tot = _run_gpu(gm, U0, 6, dts=dts)
        outs[v] = U.cpu()
    for form in forms:
        for v in form[1:]:
            assert torch.equal(outs[v], outs[form[0]]), v
    if precision == 4:
        assert torch.equal(outs[F32_SMEM[0]], outs[F32_STREAM[0]])
        for v in (F32_SMEM[0], F32_STREAM[0]):   # each form against the float64 oracle
            l1 = H.l1_rel_per_field(H.interior(outs[v], 16), H.interior(Uo, 16))
            assert max(l1) <= 2e-5, (v, l1)
    U = U0.to(gm.dtype).cuda().contiguous()
    before = U.clone()
    best, ms = gm.autotune(U)
    assert torch.equal(U, before)
    assert len(best) == 3 and all(0 <= b < nv for b in best)
    assert len(ms) == nv and all(len(t) == 3 and min(t) > 0 for t in ms)
    # a mixed per-axis choice
    mixed = [F32_SMEM[0], F32_STREAM[-1], F32_STREAM[0]] if precision == 4 else [1, 0, 1]
    gm.set_sweep_variants(mixed)
    U, _, _ = _run_gpu(gm, U0, 6, dts=dts)
    if precision == 8:
        assert torch.equal(U.cpu(), outs[0])
    else:
        l1 = H.l1_rel_per_field(H.interior(U.cpu(), 16), H.interior(Uo, 16))
        assert max(l1) <= 2e-5, l1


def test_sweep_opcount_mirrors_the_kernel():
    """The host operation count runs the sweep's formulas over the kernel's
    pencil ranges: its swept copy of the leaves matches a GPU step (no
    coarse-fine faces) to float32 tolerance, and its pencil counts are those
    of the three launches."""
    od = H.oracle_desc(root=(2, 2, 2), n=16, lmax=0)
    om = OM.root_mesh(od)
    gm = H.gpu_mesh_from_flags(od, [], 4)
    U0 = H.state(od, om.leaves, "blobs", count=12, seed=3).to(torch.float32).cuda().contiguous()
    gm.ghost_refresh(U0)
    dt = 2e-3
    for cycle in (0, 1):
        ops, pencils, cells, host = gm.sweep_opcount(U0, np.arange(gm.n_leaves), dt, cycle)
        U = U0.clone()
        gm.hydro_step(U, torch.full((1,), dt, dtype=torch.float64, device="cuda"), cycle)
        errs = H.l1_rel_per_field(H.interior(host, 16), H.interior(U.cpu(), 16))
        assert max(errs) < 2e-5, errs
        N, n, B = 24, 16, gm.n_leaves
        assert list(pencils) == [B * N * N, B * N * n, B * n * n]
        assert list(cells) == [p * n for p in pencils]
        per_cell = ops.sum(1) / cells
        assert np.all(per_cell > 300) and np.all(per_cell < 3000), per_cell
        assert np.all(ops > 0)


@pytest.mark.parametrize("pinned", [False, True])
def test_hydro_step_host_buffers_match_device_step(blob_amr, pinned):
    """The host-buffer entry point copies in, steps and copies out: the same
    interior state, dt_next and totals as the device call.  Page-locked
    memory is read and written by the GPU, interior cells only, its ghost
    cells left as they were; pageable memory is either copied whole or (on
    systems whose GPU reads the host page tables) handled the same way."""
    od, om, flags, U0, Uo, dts = blob_amr
    gm = H.gpu_mesh_from_flags(od, flags, 4)
    Ud = U0.to(torch.float32).cuda().contiguous()
    host = U0.to(torch.float32).contiguous().clone()
    if pinned:
        host = host.pin_memory()
        host[:, :, :4] = -7.0   # ghost planes of the host copy: neither read nor written
        marked = host[:, :, :4].clone()
    scratch = torch.empty_like(Ud)
    dtn = torch.zeros(1, dtype=torch.float64, device="cuda")
    tot = torch.zeros(5, dtype=torch.float64, device="cuda")
    for c in range(3):
        dt = float(dts[c])
        gm.hydro_step(Ud, torch.full((1,), dt, dtype=torch.float64, device="cuda"), c, dt_next=dtn, totals=tot)
        dn, th = gm.hydro_step_host(host, scratch, dt, c)
        assert dn == float(dtn.item())
        assert th == [float(x) for x in tot.cpu()]
    assert torch.equal(H.interior(host, 16), H.interior(Ud.cpu(), 16))
    if pinned:
        assert torch.equal(host[:, :, :4], marked)


@pytest.mark.parametrize("precision", [4, 8])
def test_hydro_step_cfl_matches_the_dt_next_loop(blob_amr, precision):
    """cello_hydro_step_cfl (dt from the start state, its reduction running
    alongside the refresh) against the loop of cello_hydro_step fed with the
    previous dt_next: the same states bit for bit in every exec mode, the
    same dt sequence, and totals equal to cello_reduce of each start state."""
    from paper_1810_01319_gb300 import EXEC_BATCHED, EXEC_GRAPH, EXEC_PLAIN
    od, om, flags, U0, Uo, dts = blob_amr
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    Ua, used_a, _ = _run_gpu(gm, U0, 4)
    for mode in (EXEC_PLAIN, EXEC_BATCHED, EXEC_GRAPH):
        gb = H.gpu_mesh_from_flags(od, flags, precision)
        gb.set_exec(mode)
        U = U0.to(gb.dtype).cuda().contiguous()
        dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        tot = torch.zeros(5, dtype=torch.float64, device="cuda")
        ref = torch.zeros(5, dtype=torch.float64, device="cuda")
        used = []
        for s in range(4):
            gb.reduce(U, 0.4, totals=ref)
            gb.hydro_step_cfl(U, s, 0.4, dt, totals=tot)
            torch.cuda.synchronize()
            used.append(float(dt))
            assert torch.equal(tot, ref)
        assert used == used_a
        assert torch.equal(U.cpu(), Ua.cpu()), mode
