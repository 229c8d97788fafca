#!/usr/bin/env python
"""Throughput of the hydro hot path: cell-updates/s of one full step (ghost
refresh, three PPM sweeps, coarse-fine flux correction, CFL dt and totals)
on the large blob workload: 16^3 root blocks of 32^3 cells (134M root cells)
refined to level 2 on the density slope (tau 0.3) of 512 seeded blobs,
periodic, gamma 5/3, FP32 bulk arithmetic with FP64 flux registers, dt and
totals, all leaves in one launch per phase replayed from a CUDA graph.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead
(a bounded sample of the same workload).  Under torchrun every rank runs an
independent replica (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per hydro step (FP32 batched vs FP64 plain), % of HBM roofline"
UNIT = "cell-updates/s"
WORKLOAD = dict(workload="blob-amr-large", root=[16, 16, 16], n=32, max_level=2, blobs=512, seed=0,
                tau=0.3, gamma=5.0 / 3.0, cfl=0.4, bc="periodic", precision="fp32-bulk/fp64-reductions",
                exec="graph", l2="inputs larger than L2 (state tens of GB)")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------- multi-rank
def combine_ranks(ms: float, cells: int, steps: int):
    """Whole-job throughput of independent replicas: the slowest rank's time
    (max over ranks) and the cells of all ranks.  Returns (value, ms_max).
    Runs on any initialised process group (nccl on GPUs, gloo on CPU)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return cells * steps / (ms / 1e3), ms
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(c) * steps / (float(t) / 1e3), float(t)


# ------------------------------------------------------------------ mesh
def build_workload(cfg, precision, device="cuda", chunk=1024, log=print):
    """Refine on the initial blob field to a fixpoint with the library's own
    flags and octree build; returns (mesh, state)."""
    from paper_1810_01319_gb300 import Mesh, make_desc, PERIODIC
    from workloads import ics
    root, n, lmax = cfg["root"], cfg["n"], cfg["max_level"]
    hi = tuple(r / max(root) for r in root)
    desc = make_desc(root, n, lmax, (0, 0, 0), hi, (PERIODIC,) * 3, precision, cfg["gamma"])

    def sample(mesh):
        U = mesh.empty_state(device)
        leaves = mesh.leaves.astype(np.int64)
        for s in range(0, mesh.n_leaves, chunk):
            part = ics.blobs(leaves[s:s + chunk], root, n, 4, (0, 0, 0), hi, cfg["gamma"],
                             count=cfg["blobs"], seed=cfg["seed"], device=device, chunk=256)
            U[s:s + chunk] = part.to(U.dtype)
            del part
        return U

    mesh = Mesh(desc)
    U = sample(mesh)
    for _ in range(lmax):
        mesh.ghost_refresh(U)
        flags = mesh.refine_flags(U, 0, cfg["tau"], cfg["tau"] / 4).cpu().numpy()
        flags = np.where(flags > 0, 1, 0).astype(np.int8)
        if not flags.any():
            break
        del U
        torch.cuda.empty_cache()
        mesh = Mesh(desc, mesh, flags)
        U = sample(mesh)
        log(f"[bench] refined: {mesh.n_leaves} leaves")
    return mesh, U


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(self.rows[0][1]),
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------- CPU oracle
def oracle_sample(cfg, seconds=15.0):
    """The FP64 oracle timed on a bounded sample of the same workload: a
    2^3-root-block periodic box of 32^3-cell blocks with the same blob
    density per volume, refined to level 2 on the same criterion, stepped
    until about `seconds` of CPU time.  Returns (cell-updates/s, cores, text)."""
    from oracle import hydro as OH
    from oracle import mesh as OM
    from workloads import ics
    r = 2
    od = OM.Desc(root=(r, r, r), n=cfg["n"], ghosts=4, max_level=cfg["max_level"], bc=(OM.PERIODIC,) * 3,
                 gamma=cfg["gamma"], hi=(1.0, 1.0, 1.0))
    count = max(1, int(round(cfg["blobs"] * (r / cfg["root"][0]) ** 3)))

    def st(mesh):
        return ics.blobs(mesh.leaves, od.root, od.n, 4, od.lo, od.hi, od.gamma, count=count, seed=cfg["seed"])
    mesh = OM.root_mesh(od)
    for _ in range(od.max_level):
        f = OH.refine_flags(OH.ghost_refresh(st(mesh), mesh), mesh, 0, cfg["tau"], cfg["tau"] / 4).numpy()
        f = np.where(f > 0, 1, 0).astype(np.int8)
        if not f.any():
            break
        mesh = OM.build(od, mesh, f)
    U = st(mesh)
    plan = OH.RefreshPlan(mesh)
    cf = OH.coarse_fine_faces(mesh)
    cells = mesh.n_leaves * od.n ** 3
    steps, t0 = 0, time.perf_counter()
    while True:
        dt = OH.reduce_dt_totals(U, mesh, cfg["cfl"])[0]
        U = OH.step(U, mesh, dt, steps, plan, cf=cf)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 50:
            break
    text = (f"oracle (torch float64 CPU) on a {r}^3-root sub-box of 32^3 blocks, {count} blobs, "
            f"{mesh.n_leaves} leaves to level {int(mesh.leaves[:, 0].max())}, {steps} steps")
    return cells * steps / el, torch.get_num_threads(), text


# ------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--root", type=int, default=16)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = dict(WORKLOAD)
    cfg["root"] = [args.root] * 3

    if args.impl == "reference":
        if rank != 0:
            return
        times = []
        text = cores = None
        for _ in range(args.warmup):
            oracle_sample(cfg, seconds=2.0)
        for _ in range(args.steps):
            v, cores, text = oracle_sample(cfg, seconds=8.0)
            times.append(v)
        v = statistics.median(times)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "dtype": "f64", "data": "synthetic", "config": cfg, "vs_baseline": None,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    log = (lambda *a: print(*a, file=sys.stderr)) if rank == 0 else (lambda *a: None)
    from paper_1810_01319_gb300 import EXEC_GRAPH, EXEC_PLAIN, build
    build.build()
    from paper_1810_01319_gb300 import _lib  # noqa: F401  (fails loudly if the library is missing)

    t_setup = time.time()
    mesh, U = build_workload(cfg, 4, log=log)
    log(f"[bench] workload ready in {time.time() - t_setup:.1f}s: {mesh.n_leaves} leaves, "
        f"{mesh.n_coarse_fine} coarse-fine faces")
    variant, variant_ms = mesh.autotune(U)
    log(f"[bench] autotuned sweep variant {variant}: {['%.2f' % t for t in variant_ms]} ms")
    mesh.set_exec(EXEC_GRAPH)
    cells = mesh.n_leaves * cfg["n"] ** 3
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_next = torch.zeros(1, dtype=torch.float64, device="cuda")
    totals = torch.zeros(5, dtype=torch.float64, device="cuda")
    mesh.reduce(U, cfg["cfl"], dt_next=dt)
    stream = torch.cuda.current_stream()

    cycle = 0
    for _ in range(args.warmup):
        mesh.hydro_step(U, dt, cycle, cfg["cfl"], dt_next=dt_next, totals=totals)
        dt.copy_(dt_next)
        cycle += 1
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            mesh.hydro_step(U, dt, cycle, cfg["cfl"], dt_next=dt_next, totals=totals)
            dt.copy_(dt_next)
            cycle += 1
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    value, ms = combine_ranks(ms, cells, args.steps)
    if world > 1:
        torch.distributed.barrier()
    launches_per_step = 4 + 3 + (1 if mesh.n_coarse_fine else 0)

    # per-phase times of one batched step (events between the library's launches)
    prof = mesh.profile_step(U, dt, cycle, cfg["cfl"])
    names = ["ghost_refresh", "sweep_1", "sweep_2", "sweep_3", "flux_correct", "reduce"]
    top = max(range(len(prof)), key=lambda i: prof[i])
    hbm, src = peaks()
    elem = 4
    N = cfg["n"] + 8
    ghost_cells = mesh.n_leaves * (N ** 3 - cfg["n"] ** 3)
    # algorithmic bytes per launch: each sweep reads and writes the five
    # fields of every leaf interior cell once; the refresh writes every ghost
    # cell and reads one source value for it; the reduction reads the interior
    alg_bytes = {"ghost_refresh": ghost_cells * 2 * 5 * elem, "sweep_1": cells * 2 * 5 * elem,
                 "sweep_2": cells * 2 * 5 * elem, "sweep_3": cells * 2 * 5 * elem,
                 "flux_correct": 0, "reduce": cells * 5 * elem}
    traffic_alg = alg_bytes[names[top]]
    achieved = traffic_alg / (prof[top] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": names[top], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": src, "traffic": None,
                "algorithmic_bytes_per_launch": traffic_alg, "phase_ms": dict(zip(names, prof))}

    # end to end through the public API: every step the host writes that
    # step's dt into pinned memory, it is copied to the device, the step runs,
    # and the step's result (dt_next and the five totals) is copied back to
    # pinned host memory and read by the host before the next step.  The
    # state itself stays resident in HBM across steps, as in a simulation.
    e2e = None
    if not args.no_e2e:
        dt_h = torch.empty(1, dtype=torch.float64, pin_memory=True)
        out_h = torch.empty(6, dtype=torch.float64, pin_memory=True)
        dt_host = float(dt.item())

        def e2e_step(c):
            nonlocal dt_host
            dt_h[0] = dt_host
            dt.copy_(dt_h, non_blocking=True)
            mesh.hydro_step(U, dt, c, cfg["cfl"], dt_next=dt_next, totals=totals)
            out_h[:1].copy_(dt_next, non_blocking=True)
            out_h[1:].copy_(totals, non_blocking=True)
            stream.synchronize()
            dt_host = float(out_h[0])
        for _ in range(2):
            e2e_step(cycle)
            cycle += 1
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step(cycle)
            cycle += 1
        el = time.perf_counter() - t0
        e2e = {"value": cells * args.steps * world / el, "unit": UNIT, "h2d_bytes_per_step": 8,
               "d2h_bytes_per_step": 48, "timer": "host wall clock, stream synchronised every step",
               "state_resident": True}

    # FP64 plain per-block path against FP32 batched on the 8^3-root blob box
    # (64 blobs, same blob density): the metric's comparison
    fp64 = None
    if not args.no_fp64:
        del U
        torch.cuda.empty_cache()
        sub = dict(cfg, root=[8, 8, 8], blobs=max(1, cfg["blobs"] // 8))
        rates = {}
        for prec, mode, steps in ((8, EXEC_PLAIN, 2), (4, EXEC_GRAPH, 5)):
            m2, U2 = build_workload(sub, prec, log=lambda *a: None)
            m2.autotune(U2)
            m2.set_exec(mode)
            d2 = torch.zeros(1, dtype=torch.float64, device="cuda")
            m2.reduce(U2, cfg["cfl"], dt_next=d2)
            m2.hydro_step(U2, d2, 0, cfg["cfl"])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for s in range(steps):
                m2.hydro_step(U2, d2, 1 + s, cfg["cfl"])
            b.record(stream)
            torch.cuda.synchronize()
            rates[prec] = m2.n_leaves * cfg["n"] ** 3 * steps / (a.elapsed_time(b) / 1e3)
            leaves2 = m2.n_leaves
            del U2, m2
            torch.cuda.empty_cache()
        fp64 = {"workload": "blob-amr 8^3 roots of 32^3, 64 blobs, level 2", "leaves": leaves2,
                "fp64_plain": rates[8], "fp32_batched_graph": rates[4], "ratio": rates[4] / rates[8],
                "unit": UNIT}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, cores, text = oracle_sample(cfg)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(cfg, leaves=mesh.n_leaves, cells=cells, coarse_fine_faces=mesh.n_coarse_fine,
                               sweep_variant=variant, sweep_variant_ms=variant_ms),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "fp64_plain": fp64,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk.summary(),
                "hbm_frac_algorithmic": value * 40 / (hbm * 1e9)}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
