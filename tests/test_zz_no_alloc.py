"""cello_reduce_noalloc: the CFL dt / conserved-totals reduction for callers
that cannot let the library allocate device memory at the point of use
(allocation-free stream captures, fixed up-front device budgets, runtimes
that own the device allocator).  Its scratch is a fixed array inside the
library.  Checked through the C ABI against cello_reduce on two calls in a
row, on different states, in both precisions: bit for bit, since both run
the same kernels in the same launch shape.  Collected last on purpose."""
import numpy as np
import pytest
import torch

import helpers as H
from oracle import mesh as OM

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [8, 4])
def test_noalloc_matches_reduce_on_two_calls(precision):
    od = H.oracle_desc(root=(2, 2, 2), n=16, lmax=2)
    om, flags = H.ic_refined(od, "blobs", count=24, seed=0)
    gm = H.gpu_mesh_from_flags(od, flags, precision)
    U = H.state(od, om.leaves, "blobs", count=24, seed=0).to(gm.dtype).cuda().contiguous()
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        ref_dt = torch.zeros(1, dtype=torch.float64, device="cuda")
        ref_tot = torch.zeros(5, dtype=torch.float64, device="cuda")
        gm.reduce(U, 0.4, dt_next=ref_dt, totals=ref_tot)
        na_dt = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        na_tot = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")
        gm.reduce_noalloc(U, 0.4, dt_next=na_dt, totals=na_tot)
        torch.cuda.synchronize()
        assert float(ref_dt) > 0
        # the same kernels in the same launch shape, only the scratch differs:
        # the results are bit-identical
        assert torch.equal(na_dt, ref_dt)
        assert torch.equal(na_tot, ref_tot)
        # advance the state so that the second call sees different data
        dt.copy_(ref_dt)
        gm.hydro_step(U, dt, call)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import ctypes

    from paper_1810_01319_gb300 import Mesh, _lib, make_desc
    d = make_desc((33, 32, 32), 8, 0, hi=(33 / 32, 1.0, 1.0), precision=4)
    m = Mesh(d)
    assert m.n_leaves > 32768
    small = torch.zeros(16, dtype=torch.float32, device="cuda")   # never read: the size check comes first
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    st = _lib.lib().cello_reduce_noalloc(m.handle, ctypes.c_void_p(small.data_ptr()), 0.4,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out[1:].data_ptr()), None)
    assert st == 1                                                  # CELLO_EINVAL
    assert "32768" in _lib.lib().cello_last_error().decode()
