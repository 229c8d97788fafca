"""The sharded step through the library's own kernels: leaves split into
Morton ranges (paper_1810_01319_gb300.partition), each rank with its own
mesh object (its own flux registers) and a pool whose leaves outside its
range are NaN.  A rank receives the interiors its ghost refresh reads
(cello_halo_pack on the sending rank, cello_halo_unpack on its own), runs
the refresh and its range's sweeps, receives the fine face fluxes of its
coarse-fine faces (cello_flux_pack / cello_flux_unpack), applies its flux
correction and reduces its range.  Every rank's leaves must equal the
unpartitioned cello_hydro_step bit for bit, dt_next (cfl x the min over
ranks) exactly, the totals to rounding.

Two forms: ranks emulated one after another in one process (2 and 3 ranks,
float64 and float32, periodic and outflow), and two processes on the one GPU
exchanging CPU copies of the GPU-packed buffers over gloo (no kernel of one
process waits for the other's)."""
import os
import socket

import numpy as np
import pytest
import torch

import helpers as H
from oracle import mesh as OM

pytestmark = pytest.mark.gpu

CYCLE, CFL = 1, 0.4


def _setup(precision, bc=(OM.PERIODIC,) * 3):
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=2, bc=bc)
    om, flags = H.ic_refined(od, "blobs", count=16, seed=2)
    U0 = H.state(od, om.leaves, "blobs", count=16, seed=2, abc=0.2)
    return od, om, flags, U0


def _plans(gm, ranks):
    from paper_1810_01319_gb300 import partition as P
    kind, idx, fine8 = gm.neighbour_table()
    owner = P.partition(gm.n_leaves, ranks)
    return owner, P.halo_plan(owner, kind, idx, fine8), P.flux_plan(owner, kind, fine8)


def _faces(entries):
    """flux-plan entries (fine leaf, axis, side) -> leaf * 6 + face"""
    return [f * 6 + 2 * a + (1 if s > 0 else 0) for f, a, s in entries]


def _reference(od, flags, U0, precision, dt):
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    U = U0.to(gm.dtype).cuda().contiguous()
    dtn = torch.zeros(1, dtype=torch.float64, device="cuda")
    tot = torch.zeros(5, dtype=torch.float64, device="cuda")
    gm.hydro_step(U, dt, CYCLE, CFL, dt_next=dtn, totals=tot)
    torch.cuda.synchronize()
    return U.cpu(), float(dtn), tot.cpu()


class Rank:
    def __init__(self, r, od, flags, U0, precision, owner):
        self.r = r
        self.gm = H.gpu_mesh_from_flags(od, flags, precision)
        mine = np.nonzero(owner == r)[0]
        self.lo, self.count = int(mine[0]), len(mine)
        U = torch.full(U0.shape, float("nan"), dtype=torch.float64)
        U[self.lo:self.lo + self.count] = U0[self.lo:self.lo + self.count]
        self.U = U.to(self.gm.dtype).cuda().contiguous()


def _run_in_process(od, flags, U0, precision, ranks, dt):
    gm0 = H.gpu_mesh_from_flags(od, flags, precision)
    owner, need, flux = _plans(gm0, ranks)
    R = [Rank(r, od, flags, U0, precision, owner) for r in range(ranks)]
    moved = 0
    for rk in R:                                   # interiors the refresh reads, rank s -> rank r
        for s in range(ranks):
            ids = need[rk.r][s]
            if ids:
                wire = R[s].gm.halo_pack(R[s].U, ids).cpu()
                rk.gm.halo_unpack(rk.U, ids, wire.cuda())
                moved += len(ids)
    for rk in R:
        rk.gm.hydro_step_part(rk.U, dt, CYCLE, rk.lo, rk.count, 0)
    fluxes = 0
    for rk in R:                                   # fine face fluxes of cross-rank coarse-fine faces
        for s in range(ranks):
            faces = _faces(flux[rk.r][s])
            if faces:
                wire = R[s].gm.flux_pack(faces).cpu()
                rk.gm.flux_unpack(faces, wire.cuda())
                fluxes += len(faces)
    for rk in R:
        rk.gm.hydro_step_part(rk.U, dt, CYCLE, rk.lo, rk.count, 1)
    parts = [rk.gm.reduce_part(rk.U, rk.lo, rk.count).cpu() for rk in R]
    torch.cuda.synchronize()
    dt_next = CFL * min(float(p[0]) for p in parts)
    totals = sum(p[1:] for p in parts)
    return R, dt_next, totals, moved, fluxes


@pytest.mark.parametrize("precision", [8, 4])
@pytest.mark.parametrize("ranks", [2, 3])
@pytest.mark.parametrize("bc", [(OM.PERIODIC,) * 3, (OM.OUTFLOW, OM.PERIODIC, OM.OUTFLOW)])
def test_sharded_step_matches_the_whole_step(precision, ranks, bc):
    od, om, flags, U0 = _setup(precision, bc)
    dt = torch.full((1,), 2e-3, dtype=torch.float64, device="cuda")
    Uref, dtn_ref, tot_ref = _reference(od, flags, U0, precision, dt)
    R, dtn, tot, moved, fluxes = _run_in_process(od, flags, U0, precision, ranks, dt)
    assert moved > 0 and fluxes > 0
    n = od.n
    for rk in R:
        sl = slice(rk.lo, rk.lo + rk.count)
        got = H.interior(rk.U.cpu()[sl], n)
        assert torch.equal(got, H.interior(Uref[sl], n)), f"rank {rk.r} differs"
    assert dtn == dtn_ref
    scale = float(tot_ref.abs().max())
    assert float((tot - tot_ref).abs().max()) <= 1e-14 * scale * 16


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_dir):
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        od, om, flags, U0 = _setup(8)
        dt = torch.full((1,), 2e-3, dtype=torch.float64, device="cuda")
        gm0 = H.gpu_mesh_from_flags(od, flags, 8)
        owner, need, flux = _plans(gm0, world)
        me = Rank(rank, od, flags, U0, 8, owner)
        peer = 1 - rank

        def swap(send):
            """send a CPU tensor to the peer and receive its (rank 0 sends first)."""
            n_out = torch.tensor([send.numel()], dtype=torch.int64)
            n_in = torch.zeros(1, dtype=torch.int64)
            if rank == 0:
                dist.send(n_out, peer); dist.recv(n_in, peer)
            else:
                dist.recv(n_in, peer); dist.send(n_out, peer)
            recv = torch.empty(int(n_in), dtype=send.dtype)
            if rank == 0:
                dist.send(send, peer); dist.recv(recv, peer)
            else:
                dist.recv(recv, peer); dist.send(send, peer)
            return recv

        out_ids, in_ids = need[peer][rank], need[rank][peer]
        send = me.gm.halo_pack(me.U, out_ids).cpu().reshape(-1) if out_ids else torch.zeros(0, dtype=torch.float64)
        recv = swap(send)
        if in_ids:
            me.gm.halo_unpack(me.U, in_ids, recv.cuda())
        me.gm.hydro_step_part(me.U, dt, CYCLE, me.lo, me.count, 0)
        out_f, in_f = _faces(flux[peer][rank]), _faces(flux[rank][peer])
        send = me.gm.flux_pack(out_f).cpu().reshape(-1) if out_f else torch.zeros(0, dtype=torch.float64)
        recv = swap(send)
        if in_f:
            me.gm.flux_unpack(in_f, recv.cuda())
        me.gm.hydro_step_part(me.U, dt, CYCLE, me.lo, me.count, 1)
        part = me.gm.reduce_part(me.U, me.lo, me.count).cpu()
        mn = part[:1].clone()
        dist.all_reduce(mn, op=dist.ReduceOp.MIN)
        tot = part[1:].clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        Uref, dtn_ref, tot_ref = _reference(od, flags, U0, 8, dt)
        sl = slice(me.lo, me.lo + me.count)
        ok = torch.equal(H.interior(me.U.cpu()[sl], od.n), H.interior(Uref[sl], od.n))
        ok = ok and CFL * float(mn) == dtn_ref
        ok = ok and float((tot - tot_ref).abs().max()) <= 1e-13 * float(tot_ref.abs().max())
        with open(os.path.join(result_dir, f"rank{rank}"), "w") as f:
            f.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_sharded_step_two_processes_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        assert (tmp_path / f"rank{r}").read_text() == "ok", r
