"""Method variants of the PPM sweep on the GPU against the oracle: the HLLC
interface flux and contact steepening of the density edge values (alone and
together), float64 within 1e-12 max relative per cell, float32 within 2e-5
L1 relative per field, on the Sod tube, an advected contact and a blob AMR
mesh (with coarse-fine faces), for every form of the sweep; the adjoint step
refuses both."""
import dataclasses

import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM
from workloads import ics

pytestmark = pytest.mark.gpu


def _run(gm, U0, dts, cycle0=0):
    U = U0.to(gm.dtype).cuda().contiguous()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s, d in enumerate(dts):
        dt.fill_(float(d))
        gm.hydro_step(U, dt, cycle0 + s, 0.4)
    torch.cuda.synchronize()
    return U.cpu()


@pytest.fixture(scope="module")
def sod_hllc():
    od = OM.Desc(root=(4, 2, 2), n=16, ghosts=4, max_level=0, hi=(1.0, 0.5, 0.5),
                 bc=(OM.OUTFLOW, OM.PERIODIC, OM.PERIODIC), gamma=1.4, riemann="hllc")
    om = OM.root_mesh(od)
    U0 = H.state(od, om.leaves, "sod")
    Uo, dts = OH.run(U0, om, 12, 0.4)
    return od, om, U0, Uo, dts


@pytest.fixture(scope="module")
def blob_hllc():
    od = H.oracle_desc(root=(2, 2, 2), n=16, lmax=2, riemann="hllc")
    om, flags = H.ic_refined(od, "blobs", count=24, seed=0)
    U0 = H.state(od, om.leaves, "blobs", count=24, seed=0)
    Uo, dts = OH.run(U0, om, 6, 0.4)
    assert len(OH.coarse_fine_faces(om)) > 0
    return od, om, flags, U0, Uo, dts


def test_hllc_differs_from_two_shock(blob_hllc):
    """The option is live: the same mesh and dt sequence with the two-shock
    flux gives a different state."""
    od, om, flags, U0, Uo, dts = blob_hllc
    m2 = OM.Mesh(dataclasses.replace(od, riemann="two-shock"), om.leaves)
    U2, _ = OH.run(U0, m2, 6, 0.4, dts=dts)
    assert not torch.equal(H.interior(U2, 16), H.interior(Uo, 16))


@pytest.mark.parametrize("variant", [0, 1])
def test_sod_hllc_fp64_matches_oracle(sod_hllc, variant):
    od, om, U0, Uo, dts = sod_hllc
    gm = H.gpu_mesh_from_flags(od, [], 8)
    gm.set_sweep_variant(variant)
    U = _run(gm, U0, dts)
    assert H.rel_err(H.interior(U, 16), H.interior(Uo, 16)) <= 1e-12


@pytest.mark.parametrize("variant", [0, 6, 11])
def test_sod_hllc_fp32_l1(sod_hllc, variant):
    od, om, U0, Uo, dts = sod_hllc
    gm = H.gpu_mesh_from_flags(od, [], 4)
    gm.set_sweep_variant(variant)
    U = _run(gm, U0, dts)
    assert max(H.l1_rel_per_field(H.interior(U, 16), H.interior(Uo, 16))) <= 2e-5


def test_blob_amr_hllc_fp64_matches_oracle(blob_hllc):
    od, om, flags, U0, Uo, dts = blob_hllc
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    U = _run(gm, U0, dts)
    assert H.rel_err(H.interior(U, 16), H.interior(Uo, 16)) <= 1e-12


@pytest.mark.parametrize("variant", [0, 9, 23])
def test_blob_amr_hllc_fp32_l1(blob_hllc, variant):
    od, om, flags, U0, Uo, dts = blob_hllc
    gm = H.gpu_mesh_from_flags(od, flags, 4)
    gm.set_sweep_variant(variant)
    U = _run(gm, U0, dts)
    assert max(H.l1_rel_per_field(H.interior(U, 16), H.interior(Uo, 16))) <= 2e-5


def test_adjoint_refuses_hllc(blob_hllc):
    from paper_1810_01319_gb300 import CelloError
    od, om, flags, U0, Uo, dts = blob_hllc
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    U = U0.cuda().contiguous()
    lam = torch.zeros_like(U)
    with pytest.raises(CelloError):
        gm.hydro_adjoint_step(U, lam, torch.full((1,), 1e-4, dtype=torch.float64, device="cuda"), 0)


# ------------------------------------------------------- contact steepening
@pytest.fixture(scope="module")
def contact_steep():
    """A density step at uniform pressure advected with u = 0.5 across a
    periodic box of 4 x 16 cells along x, steepening on."""
    od = OM.Desc(root=(4, 1, 1), n=16, ghosts=4, max_level=0, hi=(1.0, 0.25, 0.25), gamma=1.4, steepen=True)
    om = OM.root_mesh(od)
    x, _, _ = ics.cell_centres(om.leaves, od.root, od.n, od.ghosts, od.lo, od.hi)
    rho = torch.where((x > 0.25) & (x < 0.5), torch.full_like(x, 1.0), torch.full_like(x, 0.125))
    U0 = ics.conserved(rho, 0.5 * torch.ones_like(x), 0 * x, 0.1 * torch.ones_like(x), torch.ones_like(x), 1.4)
    dts = [0.004] * 30
    Uo, _ = OH.run(U0, om, 30, 0.4, dts=dts)
    # the oracle's steepening is live on this case
    Un, _ = OH.run(U0, OM.Mesh(dataclasses.replace(od, steepen=False), om.leaves), 30, 0.4, dts=dts)
    assert not torch.equal(Un, Uo)
    return od, om, U0, Uo, dts


@pytest.mark.parametrize("variant", [0, 1])
def test_contact_steepening_fp64_matches_oracle(contact_steep, variant):
    od, om, U0, Uo, dts = contact_steep
    gm = H.gpu_mesh_from_flags(od, [], 8)
    gm.set_sweep_variant(variant)
    U = _run(gm, U0, dts)
    assert H.rel_err(H.interior(U, 16), H.interior(Uo, 16)) <= 1e-12


@pytest.mark.parametrize("variant", [0, 6, 10, 11, 21])
def test_contact_steepening_fp32_l1(contact_steep, variant):
    od, om, U0, Uo, dts = contact_steep
    gm = H.gpu_mesh_from_flags(od, [], 4)
    gm.set_sweep_variant(variant)
    U = _run(gm, U0, dts)
    assert max(H.l1_rel_per_field(H.interior(U, 16), H.interior(Uo, 16))) <= 2e-5


@pytest.fixture(scope="module")
def blob_both():
    od = H.oracle_desc(root=(2, 2, 2), n=16, lmax=2, riemann="hllc", steepen=True)
    om, flags = H.ic_refined(od, "blobs", count=24, seed=0)
    U0 = H.state(od, om.leaves, "blobs", count=24, seed=0)
    Uo, dts = OH.run(U0, om, 6, 0.4)
    return od, om, flags, U0, Uo, dts


def test_blob_amr_hllc_steepened_fp64_matches_oracle(blob_both):
    od, om, flags, U0, Uo, dts = blob_both
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    U = _run(gm, U0, dts)
    assert H.rel_err(H.interior(U, 16), H.interior(Uo, 16)) <= 1e-12


@pytest.mark.parametrize("variant", [0, 9, 22, 23])
def test_blob_amr_hllc_steepened_fp32_l1(blob_both, variant):
    od, om, flags, U0, Uo, dts = blob_both
    gm = H.gpu_mesh_from_flags(od, flags, 4)
    gm.set_sweep_variant(variant)
    U = _run(gm, U0, dts)
    assert max(H.l1_rel_per_field(H.interior(U, 16), H.interior(Uo, 16))) <= 2e-5


def test_adjoint_refuses_steepening(contact_steep):
    from paper_1810_01319_gb300 import CelloError
    od, om, U0, Uo, dts = contact_steep
    gm = H.gpu_mesh_from_flags(od, [], 8)
    U = U0.cuda().contiguous()
    with pytest.raises(CelloError):
        gm.hydro_adjoint_step(U, torch.zeros_like(U), torch.full((1,), 1e-4, dtype=torch.float64, device="cuda"), 0)
