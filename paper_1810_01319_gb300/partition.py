"""Exchange plan of a leaf partition over several ranks (host logic of the
sharded step; every run of this library uses one GPU, so the plan is
exercised by a multi-process emulation on the CPU).

Sec. II.B: leaves are independent given their ghost layers; Sec. III runs
one octree per core with Charm++ placing the Blocks.  Here leaves are split
into contiguous ranges of the Morton order (a space-filling-curve split,
balanced by leaf count: every leaf holds n^3 cells).  Per step a rank needs,
from the other ranks,

* the interiors of every leaf its ghost refresh reads: same-level
  neighbours, the finer leaves restricted into its ghosts, the coarser leaf
  prolonged into them and that coarser leaf's face neighbours (the slopes of
  the limited prolongation reach one coarse cell further);
* the float64 face fluxes of the finer leaves on the far side of each of its
  coarse-fine faces (the flux correction replaces its coarse flux by their
  mean);
* a min over ranks of the CFL step and a sum of the conserved totals.

Inputs are the leaf count and the 27-entry neighbour table of
cello_neighbour_table (kind 0 same level, 1 coarser, 2 refined neighbour
node with its 8 children, 3 outside an outflow boundary; entry index
(dz+1)*9 + (dy+1)*3 + (dx+1); children in octant order oz*4 + oy*2 + ox).
"""
from __future__ import annotations

import numpy as np

SAME, COARSE, FINE, BOUNDARY = 0, 1, 2, 3


def face_entry(axis: int, side: int) -> int:
    """Neighbour-table entry of the face (axis, side)."""
    d = [0, 0, 0]
    d[axis] = side
    return (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1)


def partition(n_leaves: int, ranks: int) -> np.ndarray:
    """owner[b]: contiguous Morton ranges, sizes differing by at most one."""
    if ranks < 1 or n_leaves < ranks:
        raise ValueError("need at least one leaf per rank")
    bounds = [(r * n_leaves) // ranks for r in range(ranks + 1)]
    owner = np.empty(n_leaves, dtype=np.int32)
    for r in range(ranks):
        owner[bounds[r]:bounds[r + 1]] = r
    return owner


def _face_sources(kind, idx, fine8, leaf, out):
    """Leaves read through the six faces of `leaf` (the slope neighbours of
    a prolongation from it)."""
    for axis in range(3):
        for side in (-1, 1):
            e = face_entry(axis, side)
            k = kind[leaf, e]
            if k in (SAME, COARSE):
                out.add(int(idx[leaf, e]))
            elif k == FINE:
                out.update(int(c) for c in fine8[leaf, e] if c >= 0)


def refresh_sources(kind, idx, fine8, leaf) -> set:
    """Every leaf whose interior the ghost refresh of `leaf` reads."""
    out = set()
    for e in range(27):
        if e == 13:
            continue
        k = kind[leaf, e]
        if k == SAME:
            out.add(int(idx[leaf, e]))
        elif k == FINE:
            out.update(int(c) for c in fine8[leaf, e] if c >= 0)
        elif k == COARSE:
            c = int(idx[leaf, e])
            out.add(c)
            _face_sources(kind, idx, fine8, c, out)
    out.discard(leaf)
    return out


def halo_plan(owner, kind, idx, fine8):
    """need[r][s]: sorted leaves owned by rank s != r whose interiors rank r
    receives before its refresh (the send list of s to r is the same)."""
    ranks = int(owner.max()) + 1
    need = [[set() for _ in range(ranks)] for _ in range(ranks)]
    for b in range(len(owner)):
        r = int(owner[b])
        for src in refresh_sources(kind, idx, fine8, b):
            s = int(owner[src])
            if s != r:
                need[r][s].add(src)
    return [[sorted(x) for x in row] for row in need]


def flux_plan(owner, kind, fine8):
    """flux[r][s]: sorted (fine leaf, axis, side) of rank s's leaves whose
    face fluxes rank r needs for the coarse-fine faces of its leaves; side
    is the fine leaf's own face (the one facing the coarse leaf)."""
    ranks = int(owner.max()) + 1
    flux = [[set() for _ in range(ranks)] for _ in range(ranks)]
    for b in range(len(owner)):
        r = int(owner[b])
        for axis in range(3):
            for side in (-1, 1):
                e = face_entry(axis, side)
                if kind[b, e] != FINE:
                    continue
                near = 1 if side < 0 else 0          # the children's half facing leaf b
                for o in range(8):
                    if ((o >> axis) & 1) != near:
                        continue
                    f = int(fine8[b, e, o])
                    if f < 0:
                        raise ValueError("a child touching a coarse-fine face is not a leaf (2:1 balance broken)")
                    s = int(owner[f])
                    if s != r:
                        flux[r][s].add((f, axis, -side))
    return [[sorted(x) for x in row] for row in flux]
