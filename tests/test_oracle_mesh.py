"""Pins of the oracle's integer octree (Sec. II.B: array of octrees, one Block
per node): brute-force geometry on tiny meshes, balance and tiling
invariants, Morton order."""
import itertools

import numpy as np
import pytest

from oracle import mesh as M


def _desc(root=(2, 2, 1), n=8, lmax=2, bc=(M.PERIODIC, M.OUTFLOW, M.PERIODIC)):
    return M.Desc(root=root, n=n, ghosts=4, max_level=lmax, bc=bc,
                  hi=tuple(0.5 * r for r in root))


def _random_mesh(desc, seed, rounds=3):
    rng = np.random.default_rng(seed)
    mesh = M.root_mesh(desc)
    for _ in range(rounds):
        flags = rng.choice([-1, 0, 1], size=mesh.n_leaves, p=[0.3, 0.4, 0.3])
        mesh = M.build(desc, mesh, flags)
    return mesh


def _box(desc, t):
    return M._box(desc, *t)


def _overlap(desc, a, b):
    """Open boxes of nodes a and b intersect (periodic images counted)."""
    (alo, ahi), (blo, bhi) = _box(desc, a), _box(desc, b)
    for ax in range(3):
        ext = desc.root[ax] << desc.max_level
        shifts = (-ext, 0, ext) if desc.bc[ax] == M.PERIODIC else (0,)
        if not any(alo[ax] < bhi[ax] + s and blo[ax] + s < ahi[ax] for s in shifts):
            return False
    return True


def brute_neighbours(mesh):
    """Neighbour table by geometric search over all leaves."""
    d = mesh.desc
    leaves = [tuple(int(v) for v in lf) for lf in mesh.leaves]
    B = len(leaves)
    kind = np.full((B, 27), M.BOUNDARY, np.int8)
    idx = np.full((B, 27), -1, np.int32)
    fine8 = np.full((B, 27, 8), -1, np.int32)
    for b, (L, i, j, k) in enumerate(leaves):
        for e, (dx, dy, dz) in enumerate(M.DIRECTIONS):
            node = [L, i + dx, j + dy, k + dz]
            out = False
            for ax in range(3):
                nb = d.root[ax] << L
                if not 0 <= node[1 + ax] < nb:
                    if d.bc[ax] == M.OUTFLOW:
                        out = True
                    node[1 + ax] %= nb
            if out:
                continue
            node = tuple(node)
            hits = [q for q, t in enumerate(leaves) if _overlap(d, node, t)]
            lv = {leaves[q][0] for q in hits}
            if lv == {L}:
                assert len(hits) == 1
                kind[b, e], idx[b, e] = M.SAME, hits[0]
            elif lv == {L - 1}:
                assert len(hits) == 1
                kind[b, e], idx[b, e] = M.COARSE, hits[0]
            else:
                assert min(lv) > L
                kind[b, e] = M.FINE
                for o in range(8):
                    child = (L + 1, 2 * node[1] + (o & 1), 2 * node[2] + ((o >> 1) & 1), 2 * node[3] + (o >> 2))
                    eq = [q for q in hits if leaves[q] == child]
                    fine8[b, e, o] = eq[0] if eq else -1
    return kind, idx, fine8


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_neighbour_table_matches_brute_force(seed):
    desc = _desc()
    mesh = _random_mesh(desc, seed)
    k1, i1, f1 = M.neighbour_table(mesh)
    k2, i2, f2 = brute_neighbours(mesh)
    assert (k1 == k2).all() and (i1 == i2).all() and (f1 == f2).all()
    assert mesh.leaves[:, 0].max() >= 1


@pytest.mark.parametrize("seed", [3, 4])
def test_balance_and_tiling(seed):
    desc = _desc(root=(2, 1, 2), lmax=3)
    mesh = _random_mesh(desc, seed, rounds=4)
    leaves = [tuple(int(v) for v in lf) for lf in mesh.leaves]
    # 2:1 balance across faces, edges and corners (brute force over pairs)
    for a, b in itertools.combinations(leaves, 2):
        if abs(a[0] - b[0]) > 1:
            assert not M.touching(desc, a, b), (a, b)
    # leaves tile the domain: volumes add up, no two overlap
    vol = sum(8.0 ** -L for L, *_ in leaves)
    assert vol == pytest.approx(np.prod(desc.root))
    for a, b in itertools.combinations(leaves, 2):
        assert not _overlap(M.Desc(root=desc.root, n=8, ghosts=4, max_level=desc.max_level,
                                   bc=(M.OUTFLOW,) * 3, hi=desc.hi), a, b)


def test_morton_order_children_contiguous():
    desc = _desc(root=(2, 2, 2), lmax=2)
    mesh = M.build(desc, M.root_mesh(desc), [1] + [0] * 7)
    keys = [M.morton_key(desc, *map(int, t)) for t in mesh.leaves]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # the 8 children of root 0 come first, in octant order
    first = [tuple(int(v) for v in t) for t in mesh.leaves[:8]]
    assert first == [(1, o & 1, (o >> 1) & 1, o >> 2) for o in range(8)]


def test_build_refine_coarsen_balance():
    desc = M.Desc(root=(1, 1, 1), n=8, ghosts=4, max_level=3, bc=(M.PERIODIC,) * 3)
    m0 = M.root_mesh(desc)
    m1 = M.build(desc, m0, [1])
    assert m1.n_leaves == 8
    # refine one child twice -> balance forces neighbours
    m2 = M.build(desc, m1, [1] + [0] * 7)
    assert m2.n_leaves == 15
    flags = [1 if tuple(t) == (2, 0, 0, 0) else 0 for t in m2.leaves]
    m3 = M.build(desc, m2, flags)
    assert sum(1 for t in m3.leaves if t[0] == 3) == 8
    assert not M.balance_violators(m3)
    # coarsening a complete octet of -1 leaves restores the parent
    m4 = M.build(desc, m1, [-1] * 8)
    assert m4.n_leaves == 1
    # coarsening is refused where it would break balance
    flags = [-1 if t[0] == 2 else 0 for t in m2.leaves]
    m5 = M.build(desc, m2, flags)
    assert m5.n_leaves == 8


def test_adapt_skips_only_rebuilds_that_change_nothing():
    """The adapt driver skips the octree rebuild when no flag asks for
    refinement and no parent has all eight children flagged -1: on random
    meshes and flag sets, whenever it would skip, the oracle's build from
    those flags returns the same leaves."""
    from paper_1810_01319_gb300.drivers import may_change
    rng = np.random.default_rng(11)
    d = M.Desc(root=(2, 2, 2), n=8, ghosts=4, max_level=3)
    skipped = changed = 0
    for trial in range(40):
        mesh = M.root_mesh(d)
        for _ in range(3):
            mesh = M.build(d, mesh, rng.choice([0, 1], size=mesh.n_leaves, p=[0.7, 0.3]).astype(np.int8))
        p = rng.uniform(0.3, 1.0)
        flags = np.where(rng.random(mesh.n_leaves) < p, -1, 0).astype(np.int8)
        if trial % 5 == 0:
            flags[rng.integers(mesh.n_leaves)] = 1
        new = M.build(d, mesh, flags)
        same = np.array_equal(new.leaves, mesh.leaves)
        if not may_change(mesh.leaves, flags):
            skipped += 1
            assert same
        elif not same:
            changed += 1
    assert skipped > 5 and changed > 5
