"""Shared test helpers: matching oracle and GPU meshes, seeded states."""
import numpy as np
import torch

from oracle import mesh as OM
from workloads import ics


def oracle_desc(root=(2, 2, 2), n=8, lmax=2, bc=(OM.PERIODIC,) * 3, gamma=5.0 / 3.0, hi=None, riemann="two-shock",
                steepen=False, dual_energy=False):
    hi = hi or tuple(r / max(root) for r in root)
    return OM.Desc(root=tuple(root), n=n, ghosts=4, max_level=lmax, bc=tuple(bc), gamma=gamma, hi=hi,
                   riemann=riemann, steepen=steepen, dual_energy=dual_energy)


def flag_sequence(desc, rounds, seed, p_refine=0.4, p_coarsen=0.0):
    """Oracle meshes after `rounds` random flag rounds, with the flags used."""
    rng = np.random.default_rng(seed)
    mesh = OM.root_mesh(desc)
    meshes, flags = [mesh], []
    for _ in range(rounds):
        f = rng.choice([-1, 0, 1], size=mesh.n_leaves,
                       p=[p_coarsen, 1 - p_refine - p_coarsen, p_refine]).astype(np.int8)
        mesh = OM.build(desc, mesh, f)
        meshes.append(mesh)
        flags.append(f)
    return meshes, flags


RIEMANN_CODES = {"two-shock": 0, "hllc": 1}


def gpu_desc(odesc, precision):
    from paper_1810_01319_gb300 import make_desc
    return make_desc(odesc.root, odesc.n, odesc.max_level, odesc.lo, odesc.hi, odesc.bc, precision, odesc.gamma,
                     riemann=RIEMANN_CODES[odesc.riemann], steepening=int(odesc.steepen),
                     dual_energy=int(odesc.dual_energy))


def gpu_mesh_from_flags(odesc, flags, precision):
    from paper_1810_01319_gb300 import Mesh
    d = gpu_desc(odesc, precision)
    m = Mesh(d)
    for f in flags:
        m = Mesh(d, m, f)
    return m


def state(odesc, leaves, kind, **kw):
    f = getattr(ics, kind)
    if kind == "grf":
        U = f(leaves, odesc.root, odesc.n, odesc.ghosts, odesc.gamma, **kw)
    else:
        U = f(leaves, odesc.root, odesc.n, odesc.ghosts, odesc.lo, odesc.hi, odesc.gamma, **kw)
    return ics.with_internal_energy(U) if odesc.dual_energy else U


def interior(U, n, g=4):
    return U[:, :, g:g + n, g:g + n, g:g + n]


def max_rel(a, b, floor=1e-300):
    a = a.double().cpu()
    b = b.double().cpu()
    scale = torch.maximum(b.abs(), torch.full_like(b, floor))
    return float(((a - b).abs() / scale).max())


def l1_rel_per_field(a, b):
    a = a.double().cpu()
    b = b.double().cpu()
    out = []
    for f in range(a.shape[1]):
        den = float(b[:, f].abs().sum())
        out.append(float((a[:, f] - b[:, f]).abs().sum()) / max(den, 1e-300))
    return out


def ic_refined(odesc, kind, field=0, tau=0.3, tau_c=0.075, max_rounds=None, **kw):
    """Refine on the initial condition to a fixpoint (oracle flags, IC
    re-sampled on every new mesh).  Returns (oracle mesh, flag list)."""
    from oracle import hydro as OH
    mesh = OM.root_mesh(odesc)
    flags = []
    rounds = odesc.max_level if max_rounds is None else max_rounds
    for _ in range(rounds):
        U = OH.ghost_refresh(state(odesc, mesh.leaves, kind, **kw), mesh)
        f = OH.refine_flags(U, mesh, field, tau, tau_c).numpy()
        f = np.where(f > 0, 1, 0).astype(np.int8)     # no coarsening during set-up
        if not f.any():
            break
        mesh = OM.build(odesc, mesh, f)
        flags.append(f)
    return mesh, flags


def rel_err(a, b, rel_floor=1e-10):
    """Per-cell |a-b| / max(|b|, rel_floor * max|b of that field|), max over cells."""
    a = a.double().cpu()
    b = b.double().cpu()
    worst = 0.0
    for f in range(b.shape[1]):
        bf = b[:, f]
        floor = rel_floor * float(bf.abs().max()) + 1e-300
        worst = max(worst, float(((a[:, f] - bf).abs() / torch.clamp_min(bf.abs(), floor)).max()))
    return worst
