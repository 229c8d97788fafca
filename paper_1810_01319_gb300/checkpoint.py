"""Checkpoint and resume of a hydro run: the mesh description, the leaf list,
the state and the caller's counters (time, step, dt), through torch.save.
A resumed mesh is rebuilt from the saved leaves (cello_mesh_from_leaves), so
the continuation is bit-for-bit the uninterrupted run."""
from __future__ import annotations

import torch

from . import Mesh, make_desc

_DESC_FIELDS = ("root", "n", "ghosts", "max_level", "lo", "hi", "bc", "precision", "gamma", "riemann", "steepening",
                "dual_energy")


def save(path, mesh: Mesh, U, **meta):
    d = mesh.desc
    desc = {k: (list(getattr(d, k)) if k in ("root", "lo", "hi", "bc") else getattr(d, k)) for k in _DESC_FIELDS}
    torch.save({"desc": desc, "leaves": torch.from_numpy(mesh.leaves.copy()), "U": U.detach().cpu(), "meta": meta},
               path)


def load(path, device="cuda"):
    """Returns (mesh, U on device, meta)."""
    ck = torch.load(path, map_location="cpu", weights_only=False)
    d = ck["desc"]
    desc = make_desc(d["root"], d["n"], d["max_level"], d["lo"], d["hi"], d["bc"], d["precision"], d["gamma"],
                     d["ghosts"], d.get("riemann", 0), d.get("steepening", 0), d.get("dual_energy", 0))
    mesh = Mesh(desc, leaves=ck["leaves"].numpy())
    return mesh, ck["U"].to(device).contiguous(), ck["meta"]
