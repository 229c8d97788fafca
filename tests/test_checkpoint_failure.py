"""Failure detection (the device error word read by cello_check) and
checkpoint / resume (a mesh rebuilt from a saved leaf list).  The failures
are made on the host: a state with a NaN or a negative density is written
into a buffer and reduced; nothing faults the GPU."""
import numpy as np
import pytest
import torch

from tests import helpers as H


def _lib_and_desc(precision=8):
    from paper_1810_01319_gb300 import build
    build.build()
    from paper_1810_01319_gb300 import _lib, make_desc
    return _lib, make_desc((2, 2, 2), 8, 2, hi=(1.0, 1.0, 1.0), precision=precision)


@pytest.mark.parametrize("case", ["duplicate", "overlap", "gap", "range", "level"])
def test_mesh_from_leaves_rejects_bad_lists_on_host(case):
    """Host validation runs before any CUDA call, so it is checked on CPU."""
    import ctypes
    _lib, d = _lib_and_desc()
    roots = [(0, i, j, k) for k in range(2) for j in range(2) for i in range(2)]
    if case == "duplicate":
        ls = roots + [roots[0]]
    elif case == "overlap":
        ls = roots + [(1, 0, 0, 0)]
    elif case == "gap":
        ls = roots[:-1]
    elif case == "range":
        ls = roots[:-1] + [(0, 2, 1, 1)]
    else:
        ls = roots[:-1] + [(3, 0, 0, 0)]
    lv = np.ascontiguousarray(np.asarray(ls, dtype=np.int32))
    out = ctypes.c_void_p()
    rc = _lib.lib().cello_mesh_from_leaves(ctypes.byref(d), lv.ctypes.data_as(ctypes.c_void_p), len(lv),
                                           ctypes.byref(out))
    assert rc == 1 and not out.value


def _refined_mesh(precision):
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=2)
    mesh, flags = H.ic_refined(od, "blobs", count=6, seed=4)
    return od, mesh, flags, H.gpu_mesh_from_flags(od, flags, precision)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [4, 8])
def test_check_reports_bad_state(precision):
    from paper_1810_01319_gb300 import CelloError
    od, omesh, _, m = _refined_mesh(precision)
    dt = torch.float64 if precision == 8 else torch.float32
    U = H.state(od, omesh.leaves, "blobs", count=6, seed=4).to("cuda", dt)
    m.reduce(U)
    assert m.check() == 0
    for poison in ("nan", "negative_density", "negative_pressure", "inf_momentum"):
        V = U.clone()
        b = m.n_leaves // 2
        if poison == "nan":
            V[b, 4, 6, 5, 7] = float("nan")
        elif poison == "negative_density":
            V[b, 0, 5, 5, 5] = -1.0
        elif poison == "negative_pressure":
            V[b, 4, 9, 8, 4] = 0.0
        else:
            V[b, 2, 4, 4, 4] = float("inf")
        m.reduce(V)
        with pytest.raises(CelloError):
            m.check()
        assert m.check() == 0          # the word was cleared by the read
    # a ghost-zone NaN is not a leaf-interior state: no report
    V = U.clone()
    V[0, 0, 0, 0, 0] = float("nan")
    m.reduce(V)
    assert m.check() == 0
    # a step that produces a bad state reports it through its own reduction
    V = U.clone()
    V[1, 0, 4:12, 4:12, 4:12] = -1.0
    dtn = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.hydro_step(V, torch.full((1,), 1e-4, dtype=torch.float64, device="cuda"), 0, dt_next=dtn)
    with pytest.raises(CelloError):
        m.check()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [4, 8])
def test_checkpoint_resume_is_bit_exact(tmp_path, precision):
    from paper_1810_01319_gb300 import checkpoint
    od, omesh, _, m = _refined_mesh(precision)
    dt = torch.float64 if precision == 8 else torch.float32
    U = H.state(od, omesh.leaves, "blobs", count=6, seed=4).to("cuda", dt)
    step = torch.full((1,), 2e-4, dtype=torch.float64, device="cuda")
    for c in range(3):
        m.hydro_step(U, step, c)
    path = tmp_path / "ck.pt"
    checkpoint.save(path, m, U, cycle=3, t=6e-4)
    A = U.clone()
    for c in range(3, 6):
        m.hydro_step(A, step, c)
    m2, B, meta = checkpoint.load(path)
    assert meta == {"cycle": 3, "t": 6e-4}
    assert np.array_equal(m2.leaves, m.leaves)
    t1, t2 = m.neighbour_table(), m2.neighbour_table()
    for a, b in zip(t1, t2):
        assert np.array_equal(a, b)
    for c in range(meta["cycle"], 6):
        m2.hydro_step(B, step, c)
    assert torch.equal(interior(A), interior(B))


def interior(U):
    return U[:, :, 4:12, 4:12, 4:12]


@pytest.mark.gpu
def test_mesh_from_leaves_rejects_unbalanced_list():
    from paper_1810_01319_gb300 import CelloError, Mesh, make_desc
    d = make_desc((2, 2, 2), 8, 3, hi=(1.0, 1.0, 1.0), precision=8)
    ls = [(0, i, j, k) for k in range(2) for j in range(2) for i in range(2) if (i, j, k) != (0, 0, 0)]
    # refine root (0,0,0) to level 1, then its corner child twice: level 3 next to level 0 leaves
    ls += [(1, i, j, k) for k in range(2) for j in range(2) for i in range(2) if (i, j, k) != (1, 1, 1)]
    ls += [(2, i, j, k) for k in range(2, 4) for j in range(2, 4) for i in range(2, 4) if (i, j, k) != (3, 3, 3)]
    ls += [(3, i, j, k) for k in range(6, 8) for j in range(6, 8) for i in range(6, 8)]
    with pytest.raises(CelloError):
        Mesh(d, leaves=ls)
