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


# DRAM bytes (read + written) per 32^3 leaf of one sweep launch, measured by
# ncu on the 4^3-root blob box (3,970 leaves) for the same kernel form and
# position in the sweep order, keyed "axis-form-position"; the roofline's
# traffic is this times the leaves of the launch.
SWEEP_DRAM_BYTES_PER_LEAF = {"x-streaming-staged-sweep_1": 2.573e6,
                             "y-streaming-staged-sweep_2": 2.290e6, "y-streaming-sweep_2": 2.290e6,
                             "z-streaming-staged-sweep_3": 1.830e6, "z-streaming-sweep_3": 1.830e6}


def alu_peak(log=print):
    """The FP32 ALU roofline's denominator: measured FFMA lane instructions
    per second (cello_fp32_ffma_rate), and the nominal figure from the
    device's SM count x 128 FP32 lanes x the maximum SM clock."""
    from paper_1810_01319_gb300 import fp32_ffma_rate
    rate, ms = fp32_ffma_rate()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    try:
        mhz = float(subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=clocks.max.sm",
                                    "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                   timeout=20).stdout.split()[0])
    except Exception:
        mhz = None
    nominal = sms * 128 * mhz * 1e6 / 1e12 if mhz else None
    log(f"[bench] FP32 FFMA rate {rate / 1e12:.2f} T lane-instr/s measured ({ms:.2f} ms launch); "
        f"nominal {sms} SMs x 128 x {mhz} MHz = {nominal} T")
    return rate / 1e12, sms, mhz, nominal


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
    dual = int(cfg.get("dual_energy", 0))
    desc = make_desc(root, n, lmax, (0, 0, 0), hi, (PERIODIC,) * 3, precision, cfg["gamma"],
                     riemann=1 if cfg.get("riemann") == "hllc" else 0, steepening=int(cfg.get("steepening", 0)),
                     dual_energy=dual)

    def sample(mesh):
        U = mesh.empty_state(device)
        leaves = mesh.leaves.astype(np.int64)
        for s in range(0, mesh.n_leaves, chunk):
            part = ics.blobs(leaves[s:s + chunk], root, n, 4, (0, 0, 0), hi, cfg["gamma"],
                             count=cfg["blobs"], seed=cfg["seed"], device=device, chunk=256,
                             abc=cfg.get("abc", 0.0))
            if dual:
                part = ics.with_internal_energy(part)
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
def oracle_sample(cfg, seconds=15.0, single_core=False):
    """The FP64 oracle timed on a bounded sample of the same workload: a
    2^3-root-block periodic box of 32^3-cell blocks with the same blob
    density per volume, refined to level 2 on the same criterion, stepped
    until about `seconds` of CPU time on all the host threads torch uses
    (and, with single_core, one more step on one thread).  Returns
    (cell-updates/s of the median step, threads, text, 1-thread rate or None)."""
    from oracle import hydro as OH
    from oracle import mesh as OM
    from workloads import ics
    r = 2
    od = OM.Desc(root=(r, r, r), n=cfg["n"], ghosts=4, max_level=cfg["max_level"], bc=(OM.PERIODIC,) * 3,
                 gamma=cfg["gamma"], hi=(1.0, 1.0, 1.0), riemann=cfg.get("riemann", "two-shock"),
                 steepen=bool(cfg.get("steepening", 0)), dual_energy=bool(cfg.get("dual_energy", 0)))
    count = max(1, int(round(cfg["blobs"] * (r / cfg["root"][0]) ** 3)))

    def st(mesh):
        U = ics.blobs(mesh.leaves, od.root, od.n, 4, od.lo, od.hi, od.gamma, count=count, seed=cfg["seed"],
                      abc=cfg.get("abc", 0.0))
        return ics.with_internal_energy(U) if od.dual_energy else U
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

    def timed_steps(U, budget, max_steps):
        """Steps (each its own CFL reduction and step) until the time budget;
        returns (U, per-step seconds)."""
        per, t0 = [], time.perf_counter()
        while True:
            t1 = time.perf_counter()
            dt = OH.reduce_dt_totals(U, mesh, cfg["cfl"])[0]
            U = OH.step(U, mesh, dt, len(per), plan, cf=cf)
            per.append(time.perf_counter() - t1)
            if time.perf_counter() - t0 >= budget or len(per) >= max_steps:
                return U, per
    U, per = timed_steps(U, seconds, 50)
    threads = torch.get_num_threads()
    one_core = None
    if single_core:
        torch.set_num_threads(1)
        try:
            _, per1 = timed_steps(U, 0.0, 1)
        finally:
            torch.set_num_threads(threads)
        one_core = cells / statistics.median(per1)
    text = (f"oracle (torch float64 CPU) on a {r}^3-root sub-box of 32^3 blocks, {count} blobs, "
            f"{mesh.n_leaves} leaves to level {int(mesh.leaves[:, 0].max())}, {len(per)} steps on {threads} "
            f"threads (rate from the median step)" + (", then 1 step on 1 thread" if single_core else ""))
    return cells / statistics.median(per), threads, text, one_core


# ------------------------------------------------------------ Sedov, deep
SEDOV = dict(workload="sedov-deep", root=[4, 4, 4], n=16, max_level=5, E=1.0, rho0=1.0, p0=1e-5, gamma=1.4,
             tau=0.3, cfl=0.4, t_end=0.05, adapt_every=4, bc="periodic")


def _cfl_limiter(U, leaves, cfg, n):
    """Level, radius, density and pressure of the cell that sets the CFL
    step (diagnostic of the deep Sedov run; torch on the device state)."""
    from workloads import ics
    g = 4
    sl = (slice(None), slice(g, g + n), slice(g, g + n), slice(g, g + n))
    I = U[(slice(None), slice(None)) + sl[1:]].double()
    rho = I[:, 0].clamp_min(1e-10)
    vel = I[:, 1:4] / rho[:, None]
    ke = 0.5 * rho * (vel ** 2).sum(1)
    p = ((cfg["gamma"] - 1.0) * (I[:, 4] - ke)).clamp_min(1e-20)
    s = vel.abs().amax(1) + torch.sqrt(cfg["gamma"] * p / rho)
    lvl = torch.as_tensor(leaves[:, 0], device=U.device)
    dx = (1.0 / (cfg["root"][0] * n)) / (2.0 ** lvl.double())
    cand = dx.view(-1, 1, 1, 1) / s
    k = int(torch.argmin(cand))
    b = k // n ** 3
    x, y, z = ics.cell_centres(leaves[b:b + 1].astype(np.int64), cfg["root"], n, g, (0, 0, 0), (1, 1, 1),
                               device=U.device)
    c = k % n ** 3
    zi, yi, xi = c // (n * n) + g, (c // n) % n + g, c % n + g
    r = float(torch.sqrt((x[0, zi, yi, xi] - 0.5) ** 2 + (y[0, zi, yi, xi] - 0.5) ** 2 + (z[0, zi, yi, xi] - 0.5) ** 2))
    return int(leaves[b, 0]), r, float(rho.reshape(-1)[k]), float(p.reshape(-1)[k])


def sedov_run(cfg, precision, log=print, max_wall=300.0):
    """The deep-AMR Sedov-Taylor blast toward t_end with pressure-slope
    adaptation every few steps; stops at t_end or after max_wall seconds of
    wall time (the hot, rarefied centre keeps the CFL step small), and
    returns the measurements at the time reached.  Step time is timed with
    CUDA events around each hydro step only; adaptation is timed apart."""
    from paper_1810_01319_gb300 import Mesh, PERIODIC, make_desc
    from paper_1810_01319_gb300.drivers import adapt
    from workloads import ics
    root, n, lmax = cfg["root"], cfg["n"], cfg["max_level"]
    desc = make_desc(root, n, lmax, (0, 0, 0), (1, 1, 1), (PERIODIC,) * 3, precision, cfg["gamma"])

    def sample(mesh):
        return ics.sedov(mesh.leaves.astype(np.int64), root, n, 4, (0, 0, 0), (1, 1, 1), cfg["gamma"],
                         E=cfg["E"], rho0=cfg["rho0"], p0=cfg["p0"], max_level=lmax,
                         device="cuda").to(mesh.dtype).contiguous()
    mesh = Mesh(desc)
    U = sample(mesh)
    for _ in range(lmax):                       # refine on the initial condition to a fixpoint
        mesh.ghost_refresh(U)
        f = np.where(mesh.refine_flags(U, 4, cfg["tau"]).cpu().numpy() > 0, 1, 0).astype(np.int8)
        if not f.any():
            break
        mesh = Mesh(desc, mesh, f)
        U = sample(mesh)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t, steps, step_ms, cell_updates, max_leaves = 0.0, 0, 0.0, 0, mesh.n_leaves
    adapt_s = 0.0
    tuned = None
    wall = time.time()
    while t < cfg["t_end"] - 1e-15 and time.time() - wall < max_wall:
        if steps % cfg["adapt_every"] == 0:
            ta = time.time()
            new_mesh, U = adapt(mesh, U, 4, cfg["tau"])
            if new_mesh is not mesh and tuned is not None:
                new_mesh.set_sweep_variants(tuned)    # a rebuilt mesh keeps the tuned sweep variants
            mesh = new_mesh
            torch.cuda.synchronize()
            adapt_s += time.time() - ta
            if steps == 0:
                tuned = mesh.autotune(U)[0]
            max_leaves = max(max_leaves, mesh.n_leaves)
        mesh.reduce(U, cfg["cfl"], dt_next=dt)
        d = float(dt)
        if t + d > cfg["t_end"]:
            d = cfg["t_end"] - t
            dt.fill_(d)
        ev0.record()
        mesh.hydro_step(U, dt, steps, cfg["cfl"])
        ev1.record()
        ev1.synchronize()
        step_ms += ev0.elapsed_time(ev1)
        cell_updates += mesh.n_leaves * n ** 3
        t += d
        steps += 1
        if steps % 500 == 0:
            lv = mesh.leaves
            hist = np.bincount(lv[:, 0], minlength=cfg["max_level"] + 1).tolist()
            where = _cfl_limiter(U, lv, cfg, n)
            log(f"[sedov] step {steps} t={t:.3e} dt={d:.2e} leaves={mesh.n_leaves} levels={hist} "
                f"cfl-limiting cell: level {where[0]}, r={where[1]:.4f}, rho={where[2]:.3e}, p={where[3]:.3e} "
                f"step_ms={step_ms:.0f} adapt_s={adapt_s:.1f} wall={time.time() - wall:.0f}s")
    wall = time.time() - wall
    # shock radius: density-weighted mean radius of cells within 10 % of the peak density
    x, y, z = ics.cell_centres(mesh.leaves.astype(np.int64), root, n, 4, (0, 0, 0), (1, 1, 1), device="cuda")
    sl = (slice(None), slice(4, 4 + n), slice(4, 4 + n), slice(4, 4 + n))
    rho = U[:, 0].double()[sl]
    r = torch.sqrt((x[sl] - 0.5) ** 2 + (y[sl] - 0.5) ** 2 + (z[sl] - 0.5) ** 2)
    m = rho > 0.9 * rho.max()
    R = float((r[m] * rho[m]).sum() / rho[m].sum())
    peak = float(rho.max())
    del rho, r, x, y, z, m
    # FP32 batched (graph) against FP64 plain (one launch per leaf and phase)
    # on the final mesh and state: the metric's comparison on many uneven leaves
    from paper_1810_01319_gb300 import EXEC_GRAPH, EXEC_PLAIN
    rates = {}
    leaves = mesh.leaves
    for prec, mode, nsteps in ((4, EXEC_GRAPH, 6), (8, EXEC_PLAIN, 2)):
        d2 = make_desc(root, n, lmax, (0, 0, 0), (1, 1, 1), (PERIODIC,) * 3, prec, cfg["gamma"])
        m2 = Mesh(d2, leaves=leaves)
        if prec == 4 and tuned is not None:
            m2.set_sweep_variants(tuned)
        m2.set_exec(mode)
        U2 = U.to(m2.dtype).contiguous()
        d = torch.zeros(1, dtype=torch.float64, device="cuda")
        m2.reduce(U2, cfg["cfl"], dt_next=d)
        m2.hydro_step(U2, d, steps, cfg["cfl"])
        ev0.record()
        for k in range(nsteps):
            m2.hydro_step(U2, d, steps + 1 + k, cfg["cfl"])
        ev1.record()
        ev1.synchronize()
        rates[prec] = m2.n_leaves * n ** 3 * nsteps / (ev0.elapsed_time(ev1) / 1e3)
        del U2, m2
        torch.cuda.empty_cache()
    return {"steps": steps, "t": t, "reached_t_end": t >= cfg["t_end"] - 1e-15, "leaves_final": mesh.n_leaves,
            "final_mesh_fp32_batched": rates[4], "final_mesh_fp64_plain": rates[8],
            "final_mesh_ratio": rates[4] / rates[8],
            "leaves_max": max_leaves, "cell_updates": cell_updates, "step_ms_total": step_ms,
            "adapt_s_total": adapt_s, "wall_s": wall, "value": cell_updates / (step_ms / 1e3),
            "shock_radius": R, "peak_density": peak}


# ------------------------------------------------------- end to end, host
def host_bytes_available():
    """Bytes this process may still allocate on the host: the smaller of
    MemAvailable and the cgroup's limit minus its usage."""
    avail = None
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for lim_f, use_f in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                         ("/sys/fs/cgroup/memory/memory.limit_in_bytes", "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            lim = open(lim_f).read().strip()
            use = int(open(use_f).read().strip())
            if lim != "max" and int(lim) < (1 << 60):
                room = int(lim) - use
                avail = room if avail is None else min(avail, room)
            break
        except OSError:
            continue
    return avail or 0


def e2e_host_buffers(cfg, steps, stream, log):
    """End to end through the public API with the state in host memory, on
    the 8^3-root blob box (same blob density): the 16^3-root state (138 GB)
    cannot be held page-locked on the host next to its working copy.  Run
    before the headline workload is built, so that the device holds only
    this box."""
    from paper_1810_01319_gb300 import EXEC_GRAPH
    room = host_bytes_available()
    sub = dict(cfg, root=[8, 8, 8], blobs=max(1, cfg["blobs"] // 8))
    mesh, U = build_workload(sub, 4, log=lambda *a: None)
    workload = "blob-amr 8^3 roots of 32^3, 64 blobs, level 2"
    if room < 2 * U.numel() * U.element_size() + (16 << 30):
        log(f"[bench] e2e skipped: {room / 2**30:.0f} GiB of host memory available")
        return {"value": None, "unit": UNIT, "skipped": f"host memory ({room / 2**30:.0f} GiB available)"}
    mesh.autotune(U)
    mesh.set_exec(EXEC_GRAPH)
    m2 = mesh
    cells = mesh.n_leaves * cfg["n"] ** 3
    state_bytes = U.numel() * U.element_size()
    # what the call moves each way from page-locked memory: the interior cells (the GPU reads
    # and writes them through the buffer's device address; the step rewrites every ghost cell)
    moved_bytes = mesh.n_leaves * U.shape[1] * cfg["n"] ** 3 * U.element_size()
    cudart = torch.cuda.cudart()

    def timed(fn, reps=3):
        """Median milliseconds of fn() on the stream, CUDA events."""
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out = []
        for _ in range(reps):
            torch.cuda.synchronize()
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out)

    # the host link for the two ways of page-locking a host buffer: pageable
    # memory registered in place (cudaHostRegister) and memory allocated
    # page-locked (cudaHostAlloc, torch's pinned allocator)
    links = {}
    reg = torch.empty(U.shape, dtype=U.dtype)
    if int(cudart.cudaHostRegister(reg.data_ptr(), state_bytes, 0)) == 0:
        reg.copy_(U)
        with torch.cuda.stream(stream):
            links["registered"] = (timed(lambda: U.copy_(reg, non_blocking=True)),
                                   timed(lambda: reg.copy_(U, non_blocking=True)))
        cudart.cudaHostUnregister(reg.data_ptr())
    del reg
    host = torch.empty(U.shape, dtype=U.dtype, pin_memory=True)
    host.copy_(U)
    torch.cuda.synchronize()
    dt_next = torch.zeros(1, dtype=torch.float64, device="cuda")
    mesh.reduce(U, cfg["cfl"], dt_next=dt_next)
    dt_host = float(dt_next.item())
    h2d_extra, d2h_extra = 8, 48

    # the host link and the step alone, in the same run: the per-call time
    # should be their sum
    with torch.cuda.stream(stream):
        h2d_ms = timed(lambda: U.copy_(host, non_blocking=True))
        d2h_ms = timed(lambda: host.copy_(U, non_blocking=True))
    links["allocated"] = (h2d_ms, d2h_ms)
    dt_dev = torch.full((1,), dt_host, dtype=torch.float64, device="cuda")
    step_ms = timed(lambda: mesh.hydro_step(U, dt_dev, 0, cfg["cfl"], stream=stream))
    host.copy_(U)
    for c in range(2):
        dt_host, _ = mesh.hydro_step_host(host, U, dt_host, c, cfg["cfl"], stream=stream)
    calls = []
    t0 = time.perf_counter()
    for c in range(steps):
        t1 = time.perf_counter()
        dt_host, _ = mesh.hydro_step_host(host, U, dt_host, 2 + c, cfg["cfl"], stream=stream)
        calls.append(time.perf_counter() - t1)
    el = time.perf_counter() - t0
    res = {"value": cells * steps / el, "unit": UNIT, "h2d_bytes_per_step": moved_bytes + h2d_extra,
           "d2h_bytes_per_step": moved_bytes + d2h_extra, "workload": workload, "leaves": mesh.n_leaves,
           "call": "cello_hydro_step_host (state in page-locked host memory from cudaHostAlloc; its interior "
                   f"cells, {moved_bytes / state_bytes:.0%} of the padded state, read and written by the GPU "
                   "through the buffer's device address every step)",
           "call_ms": {"min": min(calls) * 1e3, "median": statistics.median(calls) * 1e3, "max": max(calls) * 1e3},
           "timer": "host wall clock around each call, which waits for its stream",
           "link": {"h2d_ms": h2d_ms, "d2h_ms": d2h_ms, "h2d_gbs": state_bytes / h2d_ms / 1e6,
                    "d2h_gbs": state_bytes / d2h_ms / 1e6, "step_ms": step_ms,
                    "expected_call_ms": (h2d_ms + d2h_ms) * moved_bytes / state_bytes + step_ms,
                    "how": "plain copies (copy engines) of the whole page-locked buffer and one device step, "
                           "CUDA events, median of 3, in the same run just before the timed calls; the expected "
                           "call time takes the copies' rates for the bytes the call moves",
                    "by_allocation": {k: {"h2d_gbs": state_bytes / v[0] / 1e6, "d2h_gbs": state_bytes / v[1] / 1e6}
                                      for k, v in links.items()}}}
    torch.cuda.synchronize()
    del host
    if m2 is not None:
        del U, m2
        torch.cuda.empty_cache()
    return res


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
    ap.add_argument("--no-tracers", action="store_true")
    ap.add_argument("--no-poisson", action="store_true")
    ap.add_argument("--workload", default="blob-amr-large", choices=["blob-amr-large", "sedov-deep"])
    ap.add_argument("--max-wall", type=float, default=300.0, help="wall-time bound of the sedov-deep run (s)")
    ap.add_argument("--riemann", default="two-shock", choices=["two-shock", "hllc"])
    ap.add_argument("--steepening", action="store_true", help="contact steepening of the density edge values")
    ap.add_argument("--dual-energy", action="store_true", help="dual-energy formalism (a sixth field rho e)")
    ap.add_argument("--variants", default="", help="sweep variants x,y,z instead of autotuning (profiling)")
    ap.add_argument("--abc", type=float, default=0.0,
                    help="amplitude of an ABC flow added to every cell (0: blobs in a medium at rest)")
    args = ap.parse_args()

    if args.workload == "sedov-deep":
        from paper_1810_01319_gb300 import build
        build.build()
        cfg = dict(SEDOV)
        res = sedov_run(cfg, 4, log=lambda *a: print(*a, file=sys.stderr, flush=True), max_wall=args.max_wall)
        # similarity radius at the time reached, with the published energy constant for
        # gamma = 1.4 in 3-D (Kamm & Timmes 2007: E = alpha rho R^5 / t^2, alpha = 0.851072)
        R_exact = (cfg["E"] * res["t"] ** 2 / (0.851072 * cfg["rho0"])) ** 0.2
        print(json.dumps({"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": 1, "dtype": "f32",
                          "data": "synthetic", "config": cfg, "higher_is_better": True,
                          "shock_radius": res["shock_radius"], "shock_radius_similarity": R_exact,
                          "shock_radius_rel_err": res["shock_radius"] / R_exact - 1, **res}))
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = dict(WORKLOAD)
    cfg["root"] = [args.root] * 3
    if args.abc > 0.0:
        cfg["abc"] = args.abc
    if args.riemann != "two-shock" or args.steepening:
        cfg["riemann"] = args.riemann
        cfg["steepening"] = int(args.steepening)
    if args.dual_energy:
        cfg["dual_energy"] = 1

    if args.impl == "reference":
        if rank != 0:
            return
        times = []
        text = cores = None
        for _ in range(args.warmup):
            oracle_sample(cfg, seconds=2.0)
        for _ in range(args.steps):
            v, cores, text, _ = oracle_sample(cfg, seconds=8.0)
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

    # end to end through the public API with the state in host memory: every
    # step copies the whole state from page-locked host memory to the device,
    # runs the step (dt in, dt_next and totals out), and copies the state and
    # the step's result back, read by the host before the next step
    e2e = None
    if not args.no_e2e:
        e2e = e2e_host_buffers(cfg, args.steps, torch.cuda.current_stream(), log)
        torch.cuda.empty_cache()

    t_setup = time.time()
    mesh, U = build_workload(cfg, 4, log=log)
    log(f"[bench] workload ready in {time.time() - t_setup:.1f}s: {mesh.n_leaves} leaves, "
        f"{mesh.n_coarse_fine} coarse-fine faces")
    if args.variants:
        variant, variant_ms = [int(v) for v in args.variants.split(",")], None
        mesh.set_sweep_variants(variant)
        log(f"[bench] sweep variants (x, y, z) {variant} as given")
    else:
        variant, variant_ms = mesh.autotune(U)
        log(f"[bench] autotuned sweep variants (x, y, z) {variant}: "
            f"{[['%.2f' % t for t in axes] for axes in variant_ms]} ms")
    mesh.set_exec(EXEC_GRAPH)
    alu_tops, alu_sms, alu_mhz, alu_nominal = alu_peak(log)
    cells = mesh.n_leaves * cfg["n"] ** 3
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_next = torch.zeros(1, dtype=torch.float64, device="cuda")
    totals = torch.zeros(5, dtype=torch.float64, device="cuda")
    mesh.reduce(U, cfg["cfl"], dt_next=dt)
    stream = torch.cuda.current_stream()

    # each step takes its dt from the CFL reduction of its own start state
    # (cello_hydro_step_cfl: that reduction runs alongside the ghost refresh);
    # the states are those of stepping with the previous step's dt_next
    cycle = 0
    for _ in range(args.warmup):
        mesh.hydro_step_cfl(U, cycle, cfg["cfl"], dt, totals=totals)
        cycle += 1
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            mesh.hydro_step_cfl(U, cycle, cfg["cfl"], dt, totals=totals)
            cycle += 1
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    value, ms = combine_ranks(ms, cells, args.steps)
    if world > 1:
        torch.distributed.barrier()
    # kernels per step: reduction partials + finish, refresh phases X, Y, Z
    # (+ the slow faces), three sweeps, flux correction (with coarse-fine faces)
    launches_per_step = 2 + 3 + 3 + (2 if mesh.n_coarse_fine else 0)

    # algorithmic operations of the step's sweeps, counted by the library on a
    # sample of leaves (their slabs copied to the host, ghosts refreshed) and
    # scaled to the launch; then per-phase times of one batched step on the
    # same state and cycle (events between the library's launches)
    cycle += cycle % 2          # an even cycle: the sweeps run x, y, z
    sample_ids = np.unique(np.linspace(0, mesh.n_leaves - 1, 32).round().astype(np.int64))
    mesh.ghost_refresh(U)
    t_ops = time.time()
    ops, pencils, swept_cells, _ = mesh.sweep_opcount(U, sample_ids, float(dt.item()), cycle)
    log(f"[bench] operation count on {len(sample_ids)} leaves in {time.time() - t_ops:.1f}s")
    scale = mesh.n_leaves / len(sample_ids)
    prof = mesh.profile_step(U, dt, cycle, cfg["cfl"])
    names = ["ghost_refresh", "sweep_1", "sweep_2", "sweep_3", "flux_correct", "reduce"]
    top = max(range(len(prof)), key=lambda i: prof[i])
    hbm, src = peaks()
    elem = 4
    N = cfg["n"] + 8
    ghost_cells = mesh.n_leaves * (N ** 3 - cfg["n"] ** 3)
    # algorithmic bytes per launch: each sweep reads and writes the nf (five,
    # six with dual energy) fields of every leaf interior cell once; the
    # refresh writes every ghost cell and reads one source value for it; the
    # reduction reads the interior
    nf = mesh.nf
    alg_bytes = {"ghost_refresh": ghost_cells * 2 * nf * elem, "sweep_1": cells * 2 * nf * elem,
                 "sweep_2": cells * 2 * nf * elem, "sweep_3": cells * 2 * nf * elem,
                 "flux_correct": 0, "reduce": cells * nf * elem}
    phase_names = ["primitives", "slopes_and_shock_detector", "interface_values", "flatten_and_trace",
                   "riemann_flux", "update"]
    sweeps = {}
    order = [0, 1, 2] if cycle % 2 == 0 else [2, 1, 0]
    for k in range(3):
        t = prof[1 + k] / 1e3
        v = variant[order[k]]
        sweeps[f"sweep_{k + 1}"] = {
            "axis": "xyz"[order[k]], "variant": v,
            "form": {10: "streaming-staged", 11: "streaming-staged"}.get(v % 12, "streaming") if v % 12 >= 6
            else "shared-memory",
            "ms": prof[1 + k], "hbm_gbs_algorithmic": alg_bytes[f"sweep_{k + 1}"] / t / 1e9}
        if ops is not None:
            ops_launch = float(ops[k].sum()) * scale
            sweeps[f"sweep_{k + 1}"].update({
                "ops_per_launch": ops_launch, "ops_per_updated_cell": float(ops[k].sum() / swept_cells[k]),
                "ops_by_phase_per_updated_cell": {p: float(ops[k][i] / swept_cells[k])
                                                  for i, p in enumerate(phase_names)},
                "achieved_tops": ops_launch / t / 1e12})
    kname = names[top]
    if kname.startswith("sweep") and ops is not None:
        sw = sweeps[kname]
        traffic, tsrc = None, None
        key = f"{sw['axis']}-{sw['form']}-{kname}"
        if key in SWEEP_DRAM_BYTES_PER_LEAF and cfg["n"] == 32 and mesh.nf == 5:   # measured on five fields
            traffic = SWEEP_DRAM_BYTES_PER_LEAF[key] * mesh.n_leaves
            tsrc = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per leaf of the same kernel and sweep "
                    "position on the 4^3-root blob box, times the leaves of this launch")
        roofline = {"bound": "alu", "kernel": kname, "achieved": sw["achieved_tops"], "peak": alu_tops,
                    "unit": "T FP32 lane-op/s", "frac": sw["achieved_tops"] / alu_tops,
                    "peak_source": "measured: cello_fp32_ffma_rate, FP32 fused multiply-add lane instructions "
                                   "per second, 8 CTAs x 256 threads per SM, 16 independent chains each",
                    "peak_nominal": {"value": alu_nominal, "sms": alu_sms, "sm_max_mhz": alu_mhz,
                                     "formula": "SMs x 128 FP32 lanes x max SM clock"},
                    "convention": "operation-count ratio: the numerator counts every add, multiply, divide, "
                                  "square root, comparison, abs and copysign of the sweep's formulas as one "
                                  "operation, so a fused multiply-add counts two, while the peak counts one "
                                  "FFMA instruction per lane per clock; against the flop convention (an FFMA = "
                                  "2 flops, peak x 2) the same count gives half this frac",
                    "traffic": traffic, "traffic_source": tsrc,
                    "algorithmic_ops_per_launch": sw["ops_per_launch"],
                    "ops_sample": f"{len(sample_ids)} leaves evenly spaced in Morton order, scaled by "
                                  f"{mesh.n_leaves}/{len(sample_ids)}",
                    "hbm": {"achieved": sw["hbm_gbs_algorithmic"], "peak": hbm, "unit": "GB/s",
                            "frac": sw["hbm_gbs_algorithmic"] / hbm, "peak_source": src,
                            "algorithmic_bytes_per_launch": alg_bytes[kname]},
                    "sweeps": sweeps, "phase_ms": dict(zip(names, prof))}
    else:
        achieved = alg_bytes[kname] / (prof[top] / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "peak_source": src, "traffic": None,
                    "algorithmic_bytes_per_launch": alg_bytes[kname], "sweeps": sweeps,
                    "phase_ms": dict(zip(names, prof))}
    # the memory-bound phases against the HBM roofline on their algorithmic
    # bytes (the refresh: every ghost cell written once and its source read
    # once; the reduction: the interior read once)
    roofline["memory_phases"] = {
        k: {"ms": prof[names.index(k)], "algorithmic_bytes": alg_bytes[k],
            "achieved_gbs": alg_bytes[k] / (prof[names.index(k)] / 1e3) / 1e9,
            "frac": alg_bytes[k] / (prof[names.index(k)] / 1e3) / 1e9 / hbm, "peak": hbm, "peak_source": src}
        for k in ("ghost_refresh", "reduce")}


    # tracer particles (Sec. III's hydro workload carries tracers): one push of
    # 2^27 tracers spread uniformly over the box, velocities from the refreshed
    # state; particle-steps per second
    tracers = None
    if not args.no_tracers:
        npart = 1 << 27
        gen = torch.Generator(device="cuda").manual_seed(7)
        pos = torch.rand(3, npart, dtype=torch.float64, device="cuda", generator=gen)
        leaf = mesh.particles_locate(pos)
        mesh.ghost_refresh(U)
        pdt = torch.full((1,), 1e-4, dtype=torch.float64, device="cuda")
        mesh.particles_push(U, pos, leaf, pdt)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            mesh.particles_push(U, pos, leaf, pdt)
        b.record(stream)
        torch.cuda.synchronize()
        pms = a.elapsed_time(b) / 3
        # the same tracers grouped by leaf (the paper's per-Block particle batches)
        order = torch.argsort(leaf.long(), stable=True)
        pos = pos[:, order].contiguous()
        leaf = leaf[order].contiguous()
        del order
        mesh.particles_push(U, pos, leaf, pdt)
        a.record(stream)
        for _ in range(3):
            mesh.particles_push(U, pos, leaf, pdt)
        b.record(stream)
        torch.cuda.synchronize()
        pms_sorted = a.elapsed_time(b) / 3
        tracers = {"particles": npart, "push_ms": pms, "particle_steps_per_s": npart / (pms / 1e3),
                   "push_ms_grouped_by_leaf": pms_sorted,
                   "particle_steps_per_s_grouped_by_leaf": npart / (pms_sorted / 1e3),
                   "order": "uniform random positions; then the same tracers grouped by leaf"}
        del pos, leaf
        torch.cuda.empty_cache()

    # multigrid Poisson solve (mg0, the self-gravity solver of the paper's
    # uniform-grid runs) on a uniform 16^3-root mesh of 32^3 blocks: 512^3 cells
    poisson = None
    if not args.no_poisson:
        from paper_1810_01319_gb300 import Mesh, make_desc, PERIODIC
        pm = Mesh(make_desc([16, 16, 16], 32, 0, (0, 0, 0), (1, 1, 1), (PERIODIC,) * 3, 4, cfg["gamma"]))
        gen = torch.Generator(device="cuda").manual_seed(11)
        fsrc = torch.randn(pm.n_leaves, 32, 32, 32, dtype=torch.float64, device="cuda", generator=gen)
        timing = {}
        for inner in (8, 4):
            phi, _ = pm.poisson_solve(fsrc, 1, residuals=False, inner=inner)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            phi, _ = pm.poisson_solve(fsrc, 5, phi=phi, residuals=False, inner=inner)
            b.record(stream)
            torch.cuda.synchronize()
            timing[inner] = a.elapsed_time(b) / 5
        vms = timing[4]
        _, res = pm.poisson_solve(fsrc, 5, phi=phi, residuals=True, inner=4)
        pcells = 512 ** 3
        # algorithmic bytes per V-cycle: on each level four Jacobi sweeps (read
        # phi and f, write phi: 24 B per cell), the residual restriction (read
        # phi and f: 16 B) and the prolongation (read and write phi: 16 B);
        # the levels add 1/7 to the finest
        alg = 128.0 * pcells * 8.0 / 7.0
        poisson = {"grid": "512^3 (16^3 roots x 32^3, uniform, periodic)",
                   "vcycle_ms_mixed": vms, "vcycle_ms_float64": timing[8],
                   "residual_reduction_per_cycle": (res[-1] / res[0]) ** (1.0 / (len(res) - 1)),
                   "hbm_gbs_algorithmic_float64": alg / (timing[8] / 1e3) / 1e9,
                   "hbm_frac_float64": alg / (timing[8] / 1e3) / 1e9 / hbm}
        del fsrc, phi, pm
        torch.cuda.empty_cache()

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
        v, cores, text, one = oracle_sample(cfg, single_core=True)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text,
               "value_1_core": one, "host_cores_available": len(os.sched_getaffinity(0))}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(cfg, leaves=mesh.n_leaves, cells=cells, coarse_fine_faces=mesh.n_coarse_fine,
                               sweep_variant=variant, sweep_variant_ms=variant_ms,
                               step_call="cello_hydro_step_cfl (dt from the start state; its reduction alongside "
                                         "the ghost refresh)"),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "fp64_plain": fp64, "tracers": tracers, "poisson": poisson,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk.summary(),
                "hbm_frac_algorithmic": value * 40 / (hbm * 1e9)}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
