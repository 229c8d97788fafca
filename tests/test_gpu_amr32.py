"""Parity on the headline's own kernel instantiation: 32^3-cell blocks on an
AMR mesh with coarse-fine faces on every axis and on both sides of a
coarse leaf, against the float64 oracle.

Mesh: one periodic root block of 32^3 cells refined once, and one of its
eight children refined again (7 leaves at level 1, 8 at level 2).  Through
the periodic wrap the refined child touches level-1 leaves across all six
of its faces, so the step runs the n = 32 prolongation (fine ghosts from
coarse leaves), restriction (coarse ghosts from fine leaves) and flux
correction (a level-1 leaf corrected on its low and high faces along the
same axis).  State: the seeded blob field with an ABC flow in every cell
(no region at rest, flux through every coarse-fine face), gamma 5/3.

* float64: the GPU's own CFL dt sequence for 20 steps, every cell within
  1e-12 relative of the oracle (and the dt sequence within 1e-12);
* float32: 50 steps on the oracle's dt sequence, L1 relative per field
  within 2e-5, for each form of the sweep the autotuner can pick: the
  shared-memory phases, the one-cell register walk and the staged
  four-cell x walk."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM

pytestmark = pytest.mark.gpu

N_CELLS = 32
STEPS_FP64 = 20
STEPS_FP32 = 50


@pytest.fixture(scope="module")
def amr32():
    od = H.oracle_desc(root=(1, 1, 1), n=N_CELLS, lmax=2)
    flags = [np.array([1], dtype=np.int8), np.array([1, 0, 0, 0, 0, 0, 0, 0], dtype=np.int8)]
    om = OM.root_mesh(od)
    for f in flags:
        om = OM.build(od, om, f)
    assert om.n_leaves == 15 and list(np.bincount(om.leaves[:, 0])) == [0, 7, 8]
    cf = OH.coarse_fine_faces(om)
    assert sorted({(a, s) for _, a, s, _ in cf}) == [(a, s) for a in range(3) for s in (-1, 1)]
    U0 = H.state(od, om.leaves, "blobs", count=8, seed=2, abc=0.3)
    U20, dts20 = OH.run(U0, om, STEPS_FP64, 0.4)
    U50, dts30 = OH.run(U20, om, STEPS_FP32 - STEPS_FP64, 0.4, cycle0=STEPS_FP64)
    return od, om, flags, U0, U20, U50, dts20 + dts30


def _run(gm, U0, steps, dts=None, cfl=0.4):
    U = U0.to(gm.dtype).cuda().contiguous()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_next = torch.zeros(1, dtype=torch.float64, device="cuda")
    used = []
    if dts is None:
        gm.reduce(U, cfl, dt_next=dt)
    for s in range(steps):
        if dts is not None:
            dt.fill_(float(dts[s]))
        used.append(float(dt.item()))
        gm.hydro_step(U, dt, s, cfl, dt_next=dt_next)
        if dts is None:
            dt.copy_(dt_next)
    torch.cuda.synchronize()
    return U.cpu(), used


@pytest.mark.parametrize("variant", [0, 1])
def test_amr32_fp64_20_steps(amr32, variant):
    from paper_1810_01319_gb300 import EXEC_GRAPH
    od, om, flags, U0, U20, U50, dts = amr32
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    assert gm.n_coarse_fine == len(OH.coarse_fine_faces(om))
    gm.set_exec(EXEC_GRAPH)
    gm.set_sweep_variant(variant)
    U, used = _run(gm, U0, STEPS_FP64)
    assert np.allclose(used, dts[:STEPS_FP64], rtol=1e-12, atol=0)
    err = H.rel_err(H.interior(U, N_CELLS), H.interior(U20, N_CELLS))
    assert err <= 1e-12, err


# one variant of each float32 form per axis (x, y, z): shared-memory phases,
# one-cell register walk, staged four-cell x walk with one-cell y and z (8 and 6 CTAs per SM)
FP32_FORMS = {"shared-memory": [0, 0, 0], "streaming": [6, 6, 6], "streaming-staged": [22, 22, 22],
              "streaming-staged-6": [23, 20, 20]}


@pytest.mark.parametrize("form", sorted(FP32_FORMS))
def test_amr32_fp32_50_steps(amr32, form):
    from paper_1810_01319_gb300 import EXEC_GRAPH
    od, om, flags, U0, U20, U50, dts = amr32
    gm = H.gpu_mesh_from_flags(od, flags, 4)
    gm.set_exec(EXEC_GRAPH)
    gm.set_sweep_variants(FP32_FORMS[form])
    U, _ = _run(gm, U0, STEPS_FP32, dts=dts)
    l1 = H.l1_rel_per_field(H.interior(U, N_CELLS), H.interior(U50, N_CELLS))
    assert max(l1) <= 2e-5, (form, l1)
    print(f"amr32 fp32 {form}: L1 per field after {STEPS_FP32} steps {['%.2e' % v for v in l1]}")


def test_amr32_conservation(amr32):
    """Periodic mesh: the float64 totals of the float64 step are conserved to
    round-off through the coarse-fine faces."""
    od, om, flags, U0, U20, U50, dts = amr32
    gm = H.gpu_mesh_from_flags(od, flags, 8)
    U = U0.cuda().contiguous()
    t0 = torch.zeros(5, dtype=torch.float64, device="cuda")
    t1 = torch.zeros(5, dtype=torch.float64, device="cuda")
    scale = torch.zeros(5, dtype=torch.float64, device="cuda")
    gm.reduce(U, 0.4, totals=t0)
    gm.reduce(U.abs(), 0.4, totals=scale)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for s in range(10):
        dt.fill_(float(dts[s]))
        gm.hydro_step(U, dt, s, 0.4, totals=t1)
    torch.cuda.synchronize()
    assert float(((t1 - t0).abs() / scale).max()) < 1e-13
