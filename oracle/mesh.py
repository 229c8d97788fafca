"""Array-of-octrees mesh, written plainly in Python integers (oracle side).

TEST INFRASTRUCTURE ONLY: nothing in the product library imports this module.

Sec. II.B: the Cello mesh is an array of octrees (one octree per root block, so
the domain need not be a cube); every Block is one octree node and the leaf
Blocks carry the field data.  Sec. II.B also names the Refine / Restrict /
Prolong plug-ins that drive adaptation.  The paper prints no formulas for any
of this; the readings taken here are:

* A node is (L, i, j, k): level L and block index at that level, with
  i in [0, root_x * 2**L).  Parent (L-1, i>>1, ...), children
  (L+1, 2i+ox, 2j+oy, 2k+oz).
* Leaves are ordered by the Morton interleave of their lower corner expressed
  as a block index at max_level (x in the lowest bit of each triple).  Leaves
  never nest, so the key is unique.
* The neighbour table has 27 entries per leaf, one per offset
  (dx, dy, dz) in {-1,0,1}^3, entry index (dz+1)*9 + (dy+1)*3 + (dx+1).
  kind SAME (0): idx = the leaf at the same level;
  kind COARSE (1): idx = the leaf one level coarser that contains the
  neighbour node;  kind FINE (2): the neighbour node is refined, fine8 lists
  its 8 children (octant order oz*4 + oy*2 + ox) as leaf indices, -1 where a
  child is not a leaf;  kind BOUNDARY (3): the node lies outside the domain on
  an outflow axis.  Periodic axes wrap.
* 2:1 balance across faces, edges and corners: no two touching leaves differ
  by more than one level.
* Build from flags: refine +1 leaves (below max_level); coarsen complete
  sibling octets that are all -1 when the parent would not touch a leaf two
  levels finer; then refine leaves that violate balance until none does.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

PERIODIC, OUTFLOW = 0, 1
SAME, COARSE, FINE, BOUNDARY = 0, 1, 2, 3


@dataclass(frozen=True)
class Desc:
    """Mesh description: root blocks per axis, cells per block edge n, ghost
    depth, deepest level, physical box, boundary kind per axis, gamma, and
    the Riemann solver of the PPM sweeps."""
    root: tuple
    n: int
    ghosts: int
    max_level: int
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    gamma: float = 1.4
    riemann: str = "two-shock"   # interface flux: "two-shock" (CW84) or "hllc"
    steepen: bool = False        # CW84 contact steepening of the density edge values
    dual_energy: bool = False    # a sixth field rho*e, the dual-energy formalism of Bryan et al. 1995

    @property
    def nf(self) -> int:
        """Fields per cell: (rho, rho u, rho v, rho w, E), plus rho e with
        the dual-energy formalism."""
        return 6 if self.dual_energy else 5

    def dx(self, level: int) -> float:
        """Cell width at a level (cells are cubes; checked in Mesh)."""
        return (self.hi[0] - self.lo[0]) / (self.root[0] * self.n) / (1 << level)


def direction_index(dx: int, dy: int, dz: int) -> int:
    return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)


DIRECTIONS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def morton_key(desc: Desc, L: int, i: int, j: int, k: int) -> int:
    """Interleave the lower-corner block index at max_level, x lowest."""
    s = desc.max_level - L
    x, y, z = i << s, j << s, k << s
    key = 0
    for b in range(21):
        key |= ((x >> b) & 1) << (3 * b)
        key |= ((y >> b) & 1) << (3 * b + 1)
        key |= ((z >> b) & 1) << (3 * b + 2)
    return key


class Mesh:
    """Sorted leaf list plus dense per-level occupancy maps."""

    def __init__(self, desc: Desc, leaves):
        ext = [(desc.hi[a] - desc.lo[a]) / desc.root[a] for a in range(3)]
        assert abs(ext[0] - ext[1]) < 1e-15 and abs(ext[0] - ext[2]) < 1e-15, "cells must be cubes"
        assert desc.n % 2 == 0 and desc.ghosts <= desc.n // 2
        self.desc = desc
        leaves = sorted(set(tuple(int(v) for v in lf) for lf in leaves),
                        key=lambda t: morton_key(desc, *t))
        self.leaves = np.array(leaves, dtype=np.int64).reshape(-1, 4)
        self.index = {t: b for b, t in enumerate(leaves)}
        self._maps = None

    @property
    def n_leaves(self) -> int:
        return len(self.leaves)

    def blocks_per_axis(self, L: int):
        return tuple(r << L for r in self.desc.root)

    def maps(self):
        """maps[L][z, y, x] = leaf index if a leaf sits at that node,
        -1 if the node is refined (finer leaves cover it), -2 if a coarser
        leaf covers it."""
        if self._maps is None:
            d = self.desc
            maps = []
            for L in range(d.max_level + 1):
                nx, ny, nz = self.blocks_per_axis(L)
                maps.append(np.full((nz, ny, nx), -3, dtype=np.int64))
            for b, (L, i, j, k) in enumerate(self.leaves):
                L, i, j, k = int(L), int(i), int(j), int(k)
                maps[L][k, j, i] = b
                for M in range(L + 1, d.max_level + 1):
                    s = M - L
                    maps[M][k << s:(k + 1) << s, j << s:(j + 1) << s, i << s:(i + 1) << s] = -2
                for M in range(L):
                    s = L - M
                    maps[M][k >> s, j >> s, i >> s] = -1
            for m in maps:
                assert (m != -3).all(), "leaves do not tile the domain"
            self._maps = maps
        return self._maps

    def wrap(self, L: int, axis: int, v: int):
        """Block index on one axis after the boundary rule, or None outside an
        outflow boundary."""
        nb = self.desc.root[axis] << L
        if 0 <= v < nb:
            return v
        if self.desc.bc[axis] == PERIODIC:
            return v % nb
        return None


def root_mesh(desc: Desc) -> Mesh:
    nx, ny, nz = desc.root
    return Mesh(desc, [(0, i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)])


def neighbour_table(mesh: Mesh):
    """kind[B,27] int8, idx[B,27] int32, fine8[B,27,8] int32 from the dense
    level maps (see the module docstring for the encoding)."""
    B = mesh.n_leaves
    kind = np.full((B, 27), BOUNDARY, dtype=np.int8)
    idx = np.full((B, 27), -1, dtype=np.int32)
    fine8 = np.full((B, 27, 8), -1, dtype=np.int32)
    maps = mesh.maps()
    for b, (L, i, j, k) in enumerate(mesh.leaves):
        L, i, j, k = int(L), int(i), int(j), int(k)
        for e, (dx, dy, dz) in enumerate(DIRECTIONS):
            ni, nj, nk = mesh.wrap(L, 0, i + dx), mesh.wrap(L, 1, j + dy), mesh.wrap(L, 2, k + dz)
            if ni is None or nj is None or nk is None:
                continue
            m = int(maps[L][nk, nj, ni])
            if m >= 0:
                kind[b, e], idx[b, e] = SAME, m
            elif m == -2:
                c = int(maps[L - 1][nk >> 1, nj >> 1, ni >> 1])
                assert c >= 0, "2:1 balance violated"
                kind[b, e], idx[b, e] = COARSE, c
            else:
                kind[b, e] = FINE
                for o in range(8):
                    ox, oy, oz = o & 1, (o >> 1) & 1, o >> 2
                    f = int(maps[L + 1][2 * nk + oz, 2 * nj + oy, 2 * ni + ox])
                    fine8[b, e, o] = f if f >= 0 else -1
    return kind, idx, fine8


# ---------------------------------------------------------------- geometry
def _box(desc: Desc, L: int, i: int, j: int, k: int):
    """Closed box of a node in units of max-level blocks."""
    s = 1 << (desc.max_level - L)
    return (i * s, j * s, k * s), ((i + 1) * s, (j + 1) * s, (k + 1) * s)


def touching(desc: Desc, a, b) -> bool:
    """True if the closed boxes of nodes a and b intersect, counting periodic
    images.  Used by balance and by the brute-force checks."""
    (alo, ahi), (blo, bhi) = _box(desc, *a), _box(desc, *b)
    for ax in range(3):
        ext = desc.root[ax] << desc.max_level
        shifts = (-ext, 0, ext) if desc.bc[ax] == PERIODIC else (0,)
        if not any(alo[ax] <= bhi[ax] + s and blo[ax] + s <= ahi[ax] for s in shifts):
            return False
    return True


def balance_violators(mesh: Mesh):
    """Leaves that touch a leaf two or more levels finer (dense-map form:
    a touching node one level finer that is itself refined)."""
    maps = mesh.maps()
    bad = set()
    for b, (L, i, j, k) in enumerate(mesh.leaves):
        L, i, j, k = int(L), int(i), int(j), int(k)
        if L + 1 >= mesh.desc.max_level:
            continue
        for (dx, dy, dz) in DIRECTIONS:
            if (dx, dy, dz) == (0, 0, 0):
                continue
            ni, nj, nk = mesh.wrap(L, 0, i + dx), mesh.wrap(L, 1, j + dy), mesh.wrap(L, 2, k + dz)
            if ni is None or nj is None or nk is None:
                continue
            if maps[L][nk, nj, ni] != -1:
                continue
            # children of the neighbour node that touch this leaf
            for o in range(8):
                ox, oy, oz = o & 1, (o >> 1) & 1, o >> 2
                if (dx == 1 and ox != 0) or (dx == -1 and ox != 1):
                    continue
                if (dy == 1 and oy != 0) or (dy == -1 and oy != 1):
                    continue
                if (dz == 1 and oz != 0) or (dz == -1 and oz != 1):
                    continue
                if maps[L + 1][2 * nk + oz, 2 * nj + oy, 2 * ni + ox] == -1:
                    bad.add((L, i, j, k))
    return bad


def _children(t):
    L, i, j, k = t
    return [(L + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1), 2 * k + (o >> 2)) for o in range(8)]


def build(desc: Desc, prev: Mesh | None = None, flags=None) -> Mesh:
    """New mesh from the previous one and per-leaf flags (+1 refine, 0 keep,
    -1 coarsen candidate).  No previous mesh gives the root array."""
    if prev is None:
        return root_mesh(desc)
    leaves = [tuple(int(v) for v in lf) for lf in prev.leaves]
    flags = [0] * len(leaves) if flags is None else [int(f) for f in flags]
    fl = dict(zip(leaves, flags))
    refine = {t for t in leaves if fl[t] > 0 and t[0] < desc.max_level}
    cur = set(leaves)
    for t in refine:
        cur.discard(t)
        cur.update(_children(t))
    # coarsening candidates: complete octets of unrefined leaves, all -1
    parents = {}
    for t in leaves:
        if t[0] > 0:
            p = (t[0] - 1, t[1] >> 1, t[2] >> 1, t[3] >> 1)
            parents.setdefault(p, []).append(t)
    fine_after = [t for t in cur]
    coarsen = []
    for p, kids in sorted(parents.items()):
        if len(kids) != 8 or any(fl[c] >= 0 or c in refine for c in kids):
            continue
        if any(q[0] >= p[0] + 2 and touching(desc, p, q) for q in fine_after):
            continue
        coarsen.append(p)
    for p in coarsen:
        for c in _children(p):
            cur.discard(c)
        cur.add(p)
    mesh = Mesh(desc, cur)
    while True:
        bad = balance_violators(mesh)
        if not bad:
            return mesh
        cur = set(tuple(int(v) for v in lf) for lf in mesh.leaves)
        for t in bad:
            cur.discard(t)
            cur.update(_children(t))
        mesh = Mesh(desc, cur)
