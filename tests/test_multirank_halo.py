"""The exchange plan of a sharded step (paper_1810_01319_gb300.partition),
emulated on the CPU with the oracle's arithmetic: each rank holds only its
Morton range of leaves (every other leaf poisoned with NaN), receives the
interiors its ghost refresh reads and the fine face fluxes its coarse-fine
faces need, packed into flat buffers, and reduces the CFL step (min) and the
totals (sum) with the other ranks.  Its leaves must come out bit-identical
to the unpartitioned step, the step size identical, the totals equal to
rounding.  World size 2 over gloo in separate processes; three to five ranks
in one process with the buffers handed over directly."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

DT, CYCLE, CFL = 2e-3, 1, 0.4


def _setup(bc=None, dual=False):
    import helpers as H
    from oracle import mesh as OM
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=2, dual_energy=dual,
                       **({} if bc is None else {"bc": bc}))
    rng = np.random.default_rng(11)
    mesh = OM.root_mesh(od)
    for _ in range(2):
        mesh = OM.build(od, mesh, rng.choice([0, 1], size=mesh.n_leaves, p=[0.6, 0.4]))
    U0 = H.state(od, mesh.leaves, "blobs", count=12, seed=4)
    return mesh, U0


def _plans(mesh, ranks):
    from oracle import mesh as OM
    from paper_1810_01319_gb300 import partition as P
    kind, idx, fine8 = OM.neighbour_table(mesh)
    owner = P.partition(mesh.n_leaves, ranks)
    return owner, P.halo_plan(owner, kind, idx, fine8), P.flux_plan(owner, kind, fine8)


def _interior(U, n, g=4):
    return U[:, :, g:g + n, g:g + n, g:g + n]


class Rank:
    """One rank's share of the step; exchange(peer, send_buffer, recv_count)
    is the transport (gloo or an in-process hand-over)."""

    def __init__(self, r, mesh, U0, owner, need, flux):
        self.r, self.mesh, self.owner, self.need, self.flux = r, mesh, owner, need, flux
        d = mesh.desc
        self.n, self.g = d.n, d.ghosts
        self.mine = torch.from_numpy(owner == r)
        self.U = torch.full_like(U0, float("nan"))
        self.U[self.mine] = U0[self.mine]

    def pack_interiors(self, peer):
        ids = self.need[peer][self.r]
        return _interior(self.U[ids], self.n).reshape(-1).clone() if ids else torch.zeros(0, dtype=torch.float64)

    def unpack_interiors(self, peer, buf):
        ids = self.need[self.r][peer]
        if ids:
            g, n = self.g, self.n
            self.U[ids, :, g:g + n, g:g + n, g:g + n] = buf.view(len(ids), self.U.shape[1], n, n, n)

    def sweeps(self):
        from oracle import hydro as OH
        self.U = OH.ghost_refresh(self.U, self.mesh)
        assert not torch.isnan(self.U[self.mine]).any(), "a ghost source missing from the halo plan"
        self.faces, swept = {}, set()
        for axis in OH.sweep_order(CYCLE):
            self.U, self.faces[axis] = OH.sweep(self.U, self.mesh, axis, DT,
                                                 OH.transverse_rows(self.mesh, axis, swept))
            swept.add(axis)
        # a rank keeps the face fluxes of its own leaves only (those of received leaves
        # are not computed by a sharded step): the others must arrive by the flux plan
        for axis in self.faces:
            for face in self.faces[axis]:
                face[~self.mine] = float("nan")

    def pack_fluxes(self, peer):
        parts = [self.faces[a][1 if s > 0 else 0][f].reshape(-1) for f, a, s in self.flux[peer][self.r]]
        return torch.cat(parts) if parts else torch.zeros(0, dtype=torch.float64)

    def unpack_fluxes(self, peer, buf):
        entries = self.flux[self.r][peer]
        if entries:
            per = buf.numel() // len(entries)
            for k, (f, a, s) in enumerate(entries):
                face = self.faces[a][1 if s > 0 else 0]
                face[f] = buf[k * per:(k + 1) * per].view(face.shape[1:])

    def finish(self):
        from oracle import hydro as OH
        from oracle import mesh as OM
        self.U = OH.flux_correct(self.U, self.mesh, self.faces, DT)
        mine = OM.Mesh(self.mesh.desc, self.mesh.leaves[self.owner == self.r])
        dt, totals = OH.reduce_dt_totals(self.U[self.mine], mine, CFL)
        return dt, totals

    def counts(self, peer):
        n3 = self.n ** 3 * self.U.shape[1]
        face = self.n ** 2 * self.U.shape[1]
        return len(self.need[self.r][peer]) * n3, len(self.flux[self.r][peer]) * face


def _reference(bc=None, dual=False):
    from oracle import hydro as OH
    mesh, U0 = _setup(bc, dual)
    U = OH.step(U0, mesh, DT, CYCLE)
    dt, totals = OH.reduce_dt_totals(U, mesh, CFL)
    return mesh, U, dt, totals


def _worker(r, world, port, q):
    import sys
    sys.path[:0] = [os.path.dirname(os.path.abspath(__file__)), os.path.dirname(os.path.dirname(os.path.abspath(__file__)))]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=r, world_size=world)
    mesh, U0 = _setup()
    owner, need, flux = _plans(mesh, world)
    me = Rank(r, mesh, U0, owner, need, flux)

    def exchange(send, recv_count, peer):
        recv = torch.empty(recv_count, dtype=torch.float64)
        reqs = []
        if send.numel():
            reqs.append(dist.isend(send, peer))
        if recv_count:
            reqs.append(dist.irecv(recv, peer))
        for w in reqs:
            w.wait()
        return recv

    peer = 1 - r
    me.unpack_interiors(peer, exchange(me.pack_interiors(peer), me.counts(peer)[0], peer))
    me.sweeps()
    me.unpack_fluxes(peer, exchange(me.pack_fluxes(peer), me.counts(peer)[1], peer))
    dt, totals = me.finish()
    dtt = torch.tensor([dt], dtype=torch.float64)
    dist.all_reduce(dtt, op=dist.ReduceOp.MIN)
    dist.all_reduce(totals, op=dist.ReduceOp.SUM)
    q.put((r, me.U[me.mine].clone(), float(dtt), totals.clone(), len(need[r][peer]), len(flux[r][peer])))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _random_mesh(seed, bc):
    import helpers as H
    from oracle import mesh as OM
    od = H.oracle_desc(root=(2, 3, 2), n=8, lmax=2, bc=bc)
    rng = np.random.default_rng(seed)
    mesh = OM.root_mesh(od)
    for _ in range(2):
        mesh = OM.build(od, mesh, rng.choice([-1, 0, 1], size=mesh.n_leaves, p=[0.2, 0.4, 0.4]))
    return mesh


@pytest.mark.parametrize("seed,ranks,bc", [(0, 2, (0, 0, 0)), (1, 3, (1, 0, 0)), (2, 5, (0, 1, 1)),
                                           (3, 7, (0, 0, 0))])
def test_halo_and_flux_plans_cover_the_refresh(seed, ranks, bc):
    """Every ghost source of a leaf is itself or in its rank's receive list
    (checked against the oracle's own refresh plan, source by source), on
    seeded random meshes of non-cubic root arrays split over 2 to 7 ranks."""
    from oracle import hydro as OH
    mesh = _random_mesh(seed, bc)
    owner, need, flux = _plans(mesh, ranks)
    plan = OH.RefreshPlan(mesh)
    N3 = plan.N3
    per_leaf = plan.nf * N3
    leaf_of = lambda flat: flat // per_leaf
    srcs = [(plan.copy_d, plan.copy_s.view(-1, 1)), (plan.rst_d, plan.rst_s), (plan.pro_d, plan.pro_c.view(-1, 1))]
    checked = 0
    for dst, src in srcs:
        for d, s in zip(leaf_of(dst).tolist(), leaf_of(src).tolist()):
            r = int(owner[d])
            for b in s:
                assert owner[b] == r or b in need[r][int(owner[b])]
                checked += 1
    # slope neighbours of the prolongations: one source (mode 0) or the 8 restricted children (mode 1)
    for d, nb, modes in zip(leaf_of(plan.pro_d).tolist(), leaf_of(plan.pro_nb).tolist(), plan.pro_mode.tolist()):
        r = int(owner[d])
        for row, mode in zip(nb, modes):
            for b in (row if mode == 1 else row[:1]):
                assert owner[b] == r or b in need[r][int(owner[b])]
                checked += 1
    assert checked > 1000
    assert sum(len(x) for row in flux for x in row) > 0


def test_sharded_step_gloo_world2():
    mesh, Uref, dtref, totref = _reference()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    owner = _plans(mesh, 2)[0]
    n = mesh.desc.n
    for r, Ur, dt, totals, nhalo, nflux in out:
        assert nhalo > 0 and nflux > 0          # the split cuts same-level and coarse-fine faces
        assert torch.equal(_interior(Ur, n), _interior(Uref[torch.from_numpy(owner == r)], n))
        assert dt == dtref
        assert torch.allclose(totals, totref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("nranks,bc,dual", [(3, None, False), (4, (1, 0, 1), False), (5, None, True)],
                         ids=["3-periodic", "4-outflow-xz", "5-dual-energy"])
def test_sharded_step_in_process(nranks, bc, dual):
    """Several ranks in one process, buffers handed over directly; with
    outflow faces (no neighbour behind them) and with the sixth field of
    the dual-energy formalism."""
    mesh, Uref, dtref, totref = _reference(bc, dual)
    _, U0 = _setup(bc, dual)
    owner, need, flux = _plans(mesh, nranks)
    ranks = [Rank(r, mesh, U0, owner, need, flux) for r in range(nranks)]
    for me in ranks:
        for peer in range(nranks):
            if peer != me.r:
                me.unpack_interiors(peer, ranks[peer].pack_interiors(me.r))
    for me in ranks:
        me.sweeps()
    for me in ranks:
        for peer in range(nranks):
            if peer != me.r:
                me.unpack_fluxes(peer, ranks[peer].pack_fluxes(me.r))
    res = [me.finish() for me in ranks]
    n = mesh.desc.n
    for me in ranks:
        assert torch.equal(_interior(me.U[me.mine], n), _interior(Uref[me.mine], n))
    assert min(dt for dt, _ in res) == dtref
    assert torch.allclose(sum(t for _, t in res), totref, rtol=1e-14, atol=0)
