"""Parity at the benchmark's full size and launch configuration: the
107,605-leaf blob workload (16^3 root blocks of 32^3 cells, level 2, 512
blobs), float32 graph path with the autotuned sweep.  The oracle cannot run
the whole mesh, so
(1) sampled leaves without coarse-fine faces are stepped by the oracle from
    the GPU's refreshed blocks (a leaf's three sweeps read only its own
    padded block);
(2) sampled leaves on both sides of coarse-fine faces (coarse leaves whose
    face fluxes are corrected, fine leaves whose ghosts are prolonged) are
    refreshed by the oracle's refresh plan restricted to them, from the
    state of every leaf that plan reads, stepped by the oracle together
    with the fine leaves across their coarse-fine faces, and flux
    corrected; their refreshed ghosts and their stepped interiors are
    compared with the GPU's;
(3) conservation of the float64 totals is checked on the whole mesh."""
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


def test_sampled_coarse_fine_leaves_match_oracle(workload):
    """Coarse leaves with finer face neighbours (two per coarse level) and
    fine leaves with a coarser face neighbour (two per fine level): the
    GPU's refreshed ghosts within 1e-6 of each field's largest magnitude on
    the leaf (float32 restriction and prolongation of float32 data against
    the float64 oracle: at most a few float32 roundings of values of that
    size), and one float32 step within 2e-5 L1 relative per field of the
    oracle's step with flux correction.  The flux correction must matter:
    on the corrected cells the GPU is far closer to the corrected oracle
    than the correction itself is large."""
    cfg, mesh, U = workload
    n, g = cfg["n"], 4
    N = n + 2 * g
    leaves = mesh.leaves.astype(np.int64)
    od = OM.Desc(root=tuple(cfg["root"]), n=n, ghosts=g, max_level=cfg["max_level"], bc=(OM.PERIODIC,) * 3,
                 gamma=cfg["gamma"], hi=tuple(r / max(cfg["root"]) for r in cfg["root"]))
    om = OM.Mesh(od, leaves)
    assert np.array_equal(om.leaves, leaves)
    cf = OH.coarse_fine_faces(om)
    assert len(cf) == mesh.n_coarse_fine
    by_coarse = {}
    for face in cf:
        by_coarse.setdefault(face[0], []).append(face)
    coarse = np.array(sorted(by_coarse))
    few = np.array([len(by_coarse[b]) for b in coarse])

    def slab(rho, axis, side):
        """Interior cells within 4 of a face (rho [k, z, y, x])."""
        sl = [slice(None), slice(g, g + n), slice(g, g + n), slice(g, g + n)]
        sl[3 - axis] = slice(g + n - 4, g + n) if side > 0 else slice(g, g + 4)
        return rho[tuple(sl)]

    def busiest(cand, faces_of=None, k=2):
        """The k candidates whose density varies most (next to their
        coarse-fine faces, for coarse leaves): coarse-fine faces in gas
        still at rest carry equal coarse and fine fluxes."""
        idx = torch.as_tensor(cand, device="cuda")
        rho = U[idx, 0].float()
        if faces_of is None:
            r = rho[:, g:g + n, g:g + n, g:g + n]
            spread = (r.amax(dim=(1, 2, 3)) - r.amin(dim=(1, 2, 3))).cpu().numpy()
        else:
            spread = np.zeros(len(cand))
            for axis, side in OH.FACE_ORDER:
                r = slab(rho, axis, side)
                sp = (r.amax(dim=(1, 2, 3)) - r.amin(dim=(1, 2, 3))).cpu().numpy()
                has = np.array([(axis, side) in faces_of[b] for b in cand])
                spread = np.maximum(spread, np.where(has, sp, 0.0))
        return list(np.asarray(cand)[np.argsort(-spread, kind="stable")[:k]])

    cf_sides = {b: {(a, s) for _, a, s, _ in fs} for b, fs in by_coarse.items()}
    pick = []
    for L in (0, 1):
        pick += busiest(coarse[(leaves[coarse, 0] == L) & (few <= 2)], cf_sides)
    kind, _, _ = mesh.neighbour_table()
    face_idx = [12, 14, 10, 16, 4, 22]
    has_coarser = np.any(kind[:, face_idx] == 1, axis=1)
    for L in (1, 2):
        pick += busiest(np.nonzero(has_coarser & (leaves[:, 0] == L))[0])
    compare = sorted(set(int(b) for b in pick))
    cf_mine = [face for face in cf if face[0] in set(compare)]
    kids = {k for face in cf_mine for k, _, _ in face[3]}
    subset = sorted(set(compare) | kids)
    plan = OH.RefreshPlan(om, dest=subset)
    src = plan.leaves_read()
    cplan = plan.compact(src)
    slot = {int(b): k for k, b in enumerate(src)}

    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mesh.reduce(U, cfg["cfl"], dt_next=dt)
    before = U[torch.as_tensor(src, device="cuda")].cpu().double()
    mesh.ghost_refresh(U)
    refreshed = U[torch.as_tensor(subset, device="cuda")].cpu().double()
    mesh.hydro_step(U, dt, 0, cfg["cfl"])
    after = U[torch.as_tensor(compare, device="cuda")].cpu().double()

    Vo = cplan.apply(before)[torch.as_tensor([slot[b] for b in subset])]
    inner = torch.zeros(N, N, N, dtype=torch.bool)
    inner[g:g + n, g:g + n, g:g + n] = True
    for k in range(len(subset)):
        for f in range(5):
            o = Vo[k, f][~inner]
            d = float((refreshed[k, f][~inner] - o).abs().max())
            assert d <= 1e-6 * float(o.abs().max()), (subset[k], f, d)

    local = OM.Mesh(od, leaves[subset])
    pos = {b: k for k, b in enumerate(subset)}
    cf_local = [(pos[b], a, s, [(pos[k], o1, o2) for k, o1, o2 in kk]) for b, a, s, kk in cf_mine]
    V = Vo.clone()
    swept, faces = set(), {}
    for axis in OH.sweep_order(0):
        V, faces[axis] = OH.sweep(V, local, axis, float(dt), OH.transverse_rows(local, axis, swept))
        swept.add(axis)
    V_plain = V
    V = OH.flux_correct(V, local, faces, float(dt), cf=cf_local)
    cmp = torch.as_tensor([pos[b] for b in compare])
    l1 = H.l1_rel_per_field(H.interior(after, n), H.interior(V[cmp], n))
    assert max(l1) <= 2e-5, l1
    changed = (V[cmp] != V_plain[cmp])
    assert bool(changed.any())
    err = float((after - V[cmp]).abs()[changed].max())
    mag = float((V[cmp] - V_plain[cmp]).abs()[changed].max())
    assert err < 0.25 * mag, (err, mag)
    print(f"coarse-fine sample: {len(compare)} leaves compared, {len(subset)} stepped, {len(src)} read; "
          f"L1 per field {['%.2e' % v for v in l1]}; correction max {mag:.2e}, GPU error there {err:.2e}")


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
