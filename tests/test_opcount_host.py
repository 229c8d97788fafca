"""The host operation count of the sweep (the numerator of the sweeps' ALU
roofline in bench.py) runs the sweep's own formulas in float32 through a
counting scalar over the kernel's pencil ranges: the leaves it sweeps match
the oracle's three sweeps within the float32 bar, for the plain method and
the dual-energy formalism with either solver, and the six-field sweep costs
more operations than the five-field one on the same state."""
import ctypes

import numpy as np
import pytest
import torch

import helpers as H
from oracle import hydro as OH
from oracle import mesh as OM
from workloads import ics

DT, CYCLE = 2e-3, 0


def _lib():
    from paper_1810_01319_gb300 import build
    L = ctypes.CDLL(build.build_hostcheck())
    L.cello_hc_opcount_leaf.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 7 + [ctypes.c_double] * 2 + \
        [ctypes.c_int] * 3 + [ctypes.c_void_p]
    L.cello_hc_opcount_leaf.restype = None
    return L


def _host_step(od, mesh, U0, riemann, steepen):
    """Refresh (oracle), then the three sweeps of the step leaf by leaf
    through the operation count; returns (float32 state, ops per phase)."""
    L = _lib()
    n, g = od.n, od.ghosts
    U = OH.ghost_refresh(U0, mesh).to(torch.float32).contiguous()
    counts = np.zeros(6, dtype=np.uint64)
    swept = set()
    for axis in OH.sweep_order(CYCLE):
        (a0, a1), (b0, b1) = OH.transverse_rows(mesh, axis, swept)
        for b in range(mesh.n_leaves):
            dtdx = DT / od.dx(int(mesh.leaves[b][0]))
            L.cello_hc_opcount_leaf(ctypes.c_void_p(U[b].data_ptr()), n, g, axis, a0, a1, b0, b1, dtdx, od.gamma,
                                    1 if riemann == "hllc" else 0, int(steepen), int(od.dual_energy),
                                    counts.ctypes.data_as(ctypes.c_void_p))
        swept.add(axis)
    return U, counts


def _uniform(dual, riemann="two-shock", steepen=False):
    od = H.oracle_desc(root=(2, 2, 2), n=8, lmax=0, riemann=riemann, steepen=steepen, dual_energy=dual)
    return od, OM.root_mesh(od)


@pytest.mark.parametrize("riemann,steepen", [("two-shock", False), ("hllc", True)])
@pytest.mark.parametrize("dual", [False, True])
def test_host_sweeps_match_the_oracle_hot(dual, riemann, steepen):
    od, mesh = _uniform(dual, riemann, steepen)
    U0 = H.state(od, mesh.leaves, "blobs", count=12, seed=3)
    Uo = OH.step(U0, mesh, DT, CYCLE, flux_correction=False)
    Uh, counts = _host_step(od, mesh, U0, riemann, steepen)
    assert max(H.l1_rel_per_field(H.interior(Uh, 8), H.interior(Uo, 8))) <= 2e-5
    assert np.all(counts > 0)


def test_host_sweeps_match_the_oracle_cold_dual_energy():
    """A smooth cold flow whose pressure comes from rho e in every cell."""
    od = OM.Desc(root=(8, 1, 1), n=8, ghosts=4, max_level=0, hi=(1.0, 0.125, 0.125), gamma=5.0 / 3.0,
                 dual_energy=True)
    mesh = OM.root_mesh(od)
    x = ics.cell_centres(mesh.leaves, od.root, od.n, od.ghosts, od.lo, od.hi)[0]
    one = torch.ones_like(x)
    U0 = ics.with_internal_energy(ics.conserved(one, 1.0 + 0.5 * torch.sin(2 * np.pi * x), 0 * x, 0 * x,
                                                5e-5 * one, od.gamma)).to(torch.float32).to(torch.float64)
    assert float((H.interior(U0, 8)[:, 5] / H.interior(U0, 8)[:, 4]).max()) < OH.DE_ETA1
    Uo = OH.step(U0, mesh, DT, CYCLE, flux_correction=False)
    Uh, _ = _host_step(od, mesh, U0, "two-shock", False)
    assert max(H.l1_rel_per_field(H.interior(Uh, 8), H.interior(Uo, 8))) <= 2e-5


def test_six_field_sweep_counts_more():
    od5, mesh5 = _uniform(False)
    od6, mesh6 = _uniform(True)
    U5 = H.state(od5, mesh5.leaves, "blobs", count=12, seed=3)
    U6 = ics.with_internal_energy(U5)
    _, c5 = _host_step(od5, mesh5, U5, "two-shock", False)
    _, c6 = _host_step(od6, mesh6, U6, "two-shock", False)
    assert c6.sum() > c5.sum()
    # the five-field count per updated cell stays in the range the kernel's roofline uses
    cells = 8 * (16 * 16 + 16 * 8 + 8 * 8) * 8
    assert 300 < c5.sum() / cells < 1000
