"""Parity at the benchmark's full size and launch configuration: the
107,605-leaf blob workload (16^3 root blocks of 32^3 cells, level 2, 512
blobs), float32 graph path with the autotuned sweep.  The oracle cannot run
the whole mesh, so (1) sampled leaves are stepped by the oracle from the
GPU's refreshed blocks (a leaf's three sweeps read only its own padded
block; leaves without coarse-fine faces need no flux correction) and (2)
conservation of the float64 totals is checked on the whole mesh."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    import bench
    from paper_1810_01319_gb300 import EXEC_GRAPH
    cfg = dict(bench.WORKLOAD)
    mesh, U = bench.build_workload(cfg, 4, log=lambda *a: None)
    mesh.autotune(U)
    mesh.set_exec(EXEC_GRAPH)
    return cfg, mesh, U


def test_sampled_leaves_match_oracle(workload):
    cfg, mesh, U = workload
    n, g = cfg["n"], 4
    kind, _, _ = mesh.neighbour_table()
    face_idx = [12, 14, 10, 16, 4, 22]                  # -x, +x, -y, +y, -z, +z entries of the table
    ok = np.all((kind[:, face_idx] == 0), axis=1)
    leaves = mesh.leaves
    rng = np.random.default_rng(0)
    cand = np.nonzero(ok)[0]
    sample = np.concatenate([rng.choice(cand[leaves[cand, 0] == L], 3, replace=False)
                             for L in np.unique(leaves[cand, 0])])
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mesh.reduce(U, cfg["cfl"], dt_next=dt)
    mesh.ghost_refresh(U)
    before = U[torch.as_tensor(sample, device="cuda")].double().cpu()
    mesh.hydro_step(U, dt, 0, cfg["cfl"])
    after = U[torch.as_tensor(sample, device="cuda")].double().cpu()
    worst = 0.0
    for k, b in enumerate(sample):
        L = int(leaves[b, 0])
        od = OM.Desc(root=(16 << L, 16 << L, 16 << L), n=n, ghosts=g, max_level=0, bc=(OM.PERIODIC,) * 3,
                     gamma=cfg["gamma"])
        one = OM.Mesh(od, [(0, 0, 0, 0)])
        V = before[k:k + 1].clone()
        swept = set()
        for axis in OH.sweep_order(0):
            V, _ = OH.sweep(V, one, axis, float(dt), OH.transverse_rows(one, axis, swept))
            swept.add(axis)
        l1 = H.l1_rel_per_field(H.interior(after[k:k + 1], n), H.interior(V, n))
        worst = max(worst, max(l1))
    assert worst <= 2e-5, worst


def test_conservation_full_size(workload):
    cfg, mesh, U = workload
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    t0 = torch.zeros(5, dtype=torch.float64, device="cuda")
    t1 = torch.zeros(5, dtype=torch.float64, device="cuda")
    mesh.reduce(U, cfg["cfl"], dt_next=dt, totals=t0)
    scale = torch.zeros(5, dtype=torch.float64, device="cuda")
    mesh.reduce(U.abs(), cfg["cfl"], totals=scale)
    for s in range(3):
        mesh.hydro_step(U, dt, 1 + s, cfg["cfl"], dt_next=dt, totals=t1)
    torch.cuda.synchronize()
    drift = ((t1 - t0).abs() / scale).cpu()
    assert float(drift.max()) < 1e-6, drift
