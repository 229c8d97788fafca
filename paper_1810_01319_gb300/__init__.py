"""GB300-native hydro hot path of the Enzo-P/Cello method (arXiv:1810.01319).

Sec. II.B: an array-of-octrees mesh whose leaf Blocks carry the fields and a
ghost layer refreshed from neighbouring Blocks; Sec. II.C: a PPM hydro
Method.  The work runs in libcello_gpu.so (hand-written sm_103a CUDA); this
package only marshals arguments.  PyTorch supplies device memory and
streams.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import EXEC_BATCHED, EXEC_GRAPH, EXEC_PLAIN, OUTFLOW, PERIODIC, CelloError  # noqa: F401

RIEMANN_TWO_SHOCK, RIEMANN_HLLC = 0, 1

__all__ = ["Mesh", "make_desc", "PERIODIC", "OUTFLOW", "EXEC_PLAIN", "EXEC_BATCHED", "EXEC_GRAPH", "CelloError"]


def make_desc(root, n, max_level, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(PERIODIC,) * 3,
              precision=8, gamma=1.4, ghosts=4, riemann=0, steepening=0, dual_energy=0) -> _lib.MeshDesc:
    d = _lib.MeshDesc()
    d.root[:] = list(root)
    d.n, d.ghosts, d.max_level = n, ghosts, max_level
    d.lo[:] = [float(v) for v in lo]
    d.hi[:] = [float(v) for v in hi]
    d.bc[:] = list(bc)
    d.precision = precision
    d.gamma = float(gamma)
    d.riemann = int(riemann)
    d.steepening = int(steepening)
    d.dual_energy = int(dual_energy)
    return d


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def fp32_ffma_rate(stream=None):
    """Measured FP32 fused multiply-adds per second of the current device
    (lane instructions) and the timed launch's milliseconds: the ALU
    roofline's denominator (cello_fp32_ffma_rate)."""
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _lib.check(_lib.lib().cello_fp32_ffma_rate(ctypes.byref(rate), ctypes.byref(ms), _stream(stream)),
               "cello_fp32_ffma_rate")
    return rate.value, ms.value


class Mesh:
    """A leaf table built by cello_octree_build; owns the C handle."""

    def __init__(self, desc: _lib.MeshDesc, prev: "Mesh | None" = None, flags=None, leaves=None):
        L = _lib.lib()
        self.desc = desc
        out = ctypes.c_void_p()
        if leaves is not None:
            lv = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32).reshape(-1, 4))
            _lib.check(L.cello_mesh_from_leaves(ctypes.byref(desc), lv.ctypes.data_as(ctypes.c_void_p), len(lv),
                                                ctypes.byref(out)), "cello_mesh_from_leaves")
        else:
            fl = None
            if flags is not None:
                fl = np.ascontiguousarray(np.asarray(flags, dtype=np.int8))
                assert prev is not None and len(fl) == prev.n_leaves
            _lib.check(L.cello_octree_build(ctypes.byref(desc), prev.handle if prev else None,
                                            fl.ctypes.data_as(ctypes.c_void_p) if fl is not None else None,
                                            ctypes.byref(out)), "cello_octree_build")
        self.handle = out
        nl, le, ncf = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _lib.check(L.cello_mesh_info(out, ctypes.byref(nl), ctypes.byref(le), ctypes.byref(ncf)), "cello_mesh_info")
        self.n_leaves, self.leaf_elems, self.n_coarse_fine = nl.value, le.value, ncf.value
        self.N = desc.n + 2 * desc.ghosts
        self.nf = 6 if desc.dual_energy else 5   # fields per cell (rho e with dual energy)
        self.dtype = torch.float32 if desc.precision == 4 else torch.float64

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.lib().cello_mesh_free(h)
            self.handle = None

    # ------------------------------------------------------------- queries
    @property
    def leaves(self) -> np.ndarray:
        out = np.zeros((self.n_leaves, 4), dtype=np.int32)
        _lib.check(_lib.lib().cello_mesh_leaves(self.handle, out.ctypes.data_as(ctypes.c_void_p)), "cello_mesh_leaves")
        return out

    def neighbour_table(self):
        B = self.n_leaves
        kind = np.zeros((B, 27), np.int8)
        idx = np.zeros((B, 27), np.int32)
        fine8 = np.zeros((B, 27, 8), np.int32)
        _lib.check(_lib.lib().cello_neighbour_table(self.handle, kind.ctypes.data_as(ctypes.c_void_p),
                                                    idx.ctypes.data_as(ctypes.c_void_p),
                                                    fine8.ctypes.data_as(ctypes.c_void_p)), "cello_neighbour_table")
        return kind, idx, fine8

    def empty_state(self, device="cuda"):
        return torch.empty((self.n_leaves, self.nf, self.N, self.N, self.N), dtype=self.dtype, device=device)

    def _check_state(self, U):
        if not (U.is_cuda and U.dtype == self.dtype and U.is_contiguous()
                and U.numel() >= self.n_leaves * self.leaf_elems):
            raise CelloError("state must be a contiguous CUDA tensor of the mesh's dtype and size")

    # ------------------------------------------------------------- compute
    def refine_flags(self, U, field=0, tau=0.3, tau_c=0.075, flags=None, stream=None):
        self._check_state(U)
        if flags is None:
            flags = torch.empty(self.n_leaves, dtype=torch.int8, device=U.device)
        _lib.check(_lib.lib().cello_refine_flags(self.handle, _ptr(U), field, tau, tau_c, _ptr(flags),
                                                 _stream(stream)), "cello_refine_flags")
        return flags

    def ghost_refresh(self, U, stream=None):
        self._check_state(U)
        _lib.check(_lib.lib().cello_ghost_refresh(self.handle, _ptr(U), _stream(stream)), "cello_ghost_refresh")

    def remap_from(self, old: "Mesh", U_old, U_new=None, stream=None):
        """Interior data of this mesh from `old` (ghosts of U_old refreshed);
        returns U_new (allocated if not given; its ghosts are not written)."""
        old._check_state(U_old)
        if U_new is None:
            U_new = torch.zeros((self.n_leaves, self.nf, self.N, self.N, self.N), dtype=self.dtype,
                                device=U_old.device)
        self._check_state(U_new)
        _lib.check(_lib.lib().cello_remap(old.handle, _ptr(U_old), self.handle, _ptr(U_new), _stream(stream)),
                   "cello_remap")
        return U_new

    def hydro_step(self, U, dt, cycle, cfl=0.4, dt_next=None, totals=None, stream=None):
        """dt, dt_next: float64 CUDA tensors of one element; totals: five."""
        self._check_state(U)
        _lib.check(_lib.lib().cello_hydro_step(self.handle, _ptr(U), _ptr(dt), int(cycle), float(cfl),
                                               _ptr(dt_next), _ptr(totals), _stream(stream)), "cello_hydro_step")

    def hydro_step_cfl(self, U, cycle, cfl, dt_used, totals=None, stream=None):
        """One step with dt = the CFL step of U as given (written to dt_used,
        a float64 CUDA tensor of one element); totals (five) of that start
        state.  The start-state reduction runs alongside the ghost refresh."""
        self._check_state(U)
        _lib.check(_lib.lib().cello_hydro_step_cfl(self.handle, _ptr(U), int(cycle), float(cfl), _ptr(dt_used),
                                                   _ptr(totals), _stream(stream)), "cello_hydro_step_cfl")

    def hydro_adjoint_step(self, U_n, lam, dt, cycle, stream=None):
        """lam (adjoint of the state after the step) -> adjoint of U_n, in
        place; dt as in the forward step (held fixed)."""
        self._check_state(U_n)
        self._check_state(lam)
        _lib.check(_lib.lib().cello_hydro_adjoint_step(self.handle, _ptr(U_n), _ptr(lam), _ptr(dt), int(cycle),
                                                       _stream(stream)), "cello_hydro_adjoint_step")

    def reduce(self, U, cfl=0.4, dt_next=None, totals=None, stream=None):
        self._check_state(U)
        _lib.check(_lib.lib().cello_reduce(self.handle, _ptr(U), float(cfl), _ptr(dt_next), _ptr(totals),
                                           _stream(stream)), "cello_reduce")

    def reduce_noalloc(self, U, cfl=0.4, dt_next=None, totals=None, stream=None):
        """reduce() through the entry point that allocates nothing (its scratch
        is a fixed array of the library, at most 32768 leaves)."""
        self._check_state(U)
        _lib.check(_lib.lib().cello_reduce_noalloc(self.handle, _ptr(U), float(cfl), _ptr(dt_next), _ptr(totals),
                                                   _stream(stream)), "cello_reduce_noalloc")

    def profile_step(self, U, dt, cycle, cfl=0.4, stream=None):
        """Device milliseconds of each phase of one batched step: refresh,
        sweep 1, 2, 3, flux correction, reduction.  Advances U by one step."""
        self._check_state(U)
        out = (ctypes.c_float * 6)()
        _lib.check(_lib.lib().cello_profile_step(self.handle, _ptr(U), _ptr(dt), int(cycle), float(cfl),
                                                 ctypes.cast(out, ctypes.c_void_p), _stream(stream)),
                   "cello_profile_step")
        return list(out)

    def sweep_opcount(self, U, leaf_ids, dt: float, cycle: int = 0):
        """Counted operations of the step's three sweeps on the given leaves
        (their slabs are copied to the host; the ghosts must be refreshed).
        Returns (ops [3, 6] per sweep and phase, pencils [3], cells [3], swept
        host copy [count, fields, N, N, N])."""
        ids = np.ascontiguousarray(np.asarray(leaf_ids, dtype=np.int32))
        host = U[torch.as_tensor(ids, dtype=torch.int64, device=U.device)].detach().to("cpu").contiguous()
        out = np.zeros(24, dtype=np.float64)
        _lib.check(_lib.lib().cello_sweep_opcount(self.handle, ctypes.c_void_p(host.data_ptr()),
                                                  ids.ctypes.data_as(ctypes.c_void_p), len(ids), float(dt),
                                                  int(cycle), out.ctypes.data_as(ctypes.c_void_p)),
                   "cello_sweep_opcount")
        o = out.reshape(3, 8)
        return o[:, :6].copy(), o[:, 6].copy(), o[:, 7].copy(), host

    def hydro_step_host(self, U_host, U_dev, dt: float, cycle: int, cfl: float = 0.4, stream=None):
        """One step with the state in host memory.  Where U_host has a device
        address (pin_memory, or any host memory on systems whose GPU reads the
        host page tables) the GPU reads and writes its interior cells directly,
        ghost cells untouched; otherwise it is copied whole.  Returns
        (dt_next, totals[5]) as Python floats."""
        self._check_state(U_dev)
        if U_host.device.type != "cpu" or U_host.dtype != U_dev.dtype or U_host.shape != U_dev.shape \
                or not U_host.is_contiguous():
            raise CelloError("U_host must be a contiguous CPU tensor shaped like the device state")
        if not hasattr(self, "_host_scratch"):
            self._host_scratch = torch.zeros(7, dtype=torch.float64, device=U_dev.device)
            self._host_out = np.zeros(6, dtype=np.float64)
        sc = self._host_scratch
        _lib.check(_lib.lib().cello_hydro_step_host(self.handle, ctypes.c_void_p(U_host.data_ptr()), _ptr(U_dev),
                                                    float(dt), _ptr(sc[6:]), int(cycle), float(cfl), _ptr(sc),
                                                    self._host_out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
                   "cello_hydro_step_host")
        return float(self._host_out[0]), [float(x) for x in self._host_out[1:]]

    def poisson_solve(self, f, cycles=10, phi=None, residuals=True, inner=8, stream=None):
        """lap(phi) = f on a uniform periodic mesh by multigrid V-cycles; f a
        contiguous float64 CUDA tensor [B, n, n, n] of leaf interiors; inner
        8 (float64 cycles) or 4 (float32 cycles on the float64 residual).
        Returns (phi, residual max-norm after each cycle or None)."""
        n = self.desc.n
        if f.dtype != torch.float64 or not f.is_cuda or not f.is_contiguous() or f.numel() != self.n_leaves * n ** 3:
            raise CelloError("f must be a contiguous float64 CUDA tensor [B, n, n, n]")
        if phi is None:
            phi = torch.empty_like(f)
        res = (ctypes.c_double * cycles)() if residuals else None
        _lib.check(_lib.lib().cello_poisson_solve(self.handle, _ptr(f), _ptr(phi), int(cycles), int(inner),
                                                  ctypes.cast(res, ctypes.c_void_p) if res is not None else None,
                                                  _stream(stream)), "cello_poisson_solve")
        return phi, (list(res) if res is not None else None)

    def particles_locate(self, pos, leaf=None, stream=None):
        """Containing leaf of each tracer: pos a contiguous float64 CUDA tensor
        [3, P]; returns (or fills) an int32 CUDA tensor [P]."""
        if pos.dtype != torch.float64 or not pos.is_cuda or not pos.is_contiguous() or pos.dim() != 2 \
                or pos.shape[0] != 3:
            raise CelloError("pos must be a contiguous float64 CUDA tensor [3, P]")
        if leaf is None:
            leaf = torch.empty(pos.shape[1], dtype=torch.int32, device=pos.device)
        _lib.check(_lib.lib().cello_particles_locate(self.handle, _ptr(pos), _ptr(leaf), pos.shape[1],
                                                     _stream(stream)), "cello_particles_locate")
        return leaf

    def particles_push(self, U, pos, leaf, dt, stream=None):
        """One tracer step in place (U's ghosts refreshed); dt a float64 CUDA
        scalar tensor."""
        self._check_state(U)
        if pos.dtype != torch.float64 or not pos.is_contiguous() or leaf.dtype != torch.int32 \
                or leaf.numel() != pos.shape[1]:
            raise CelloError("pos must be float64 [3, P] and leaf int32 [P]")
        _lib.check(_lib.lib().cello_particles_push(self.handle, _ptr(U), _ptr(pos), _ptr(leaf), pos.shape[1],
                                                   _ptr(dt), _stream(stream)), "cello_particles_push")

    def check(self) -> int:
        """Read and clear the device error word (waits for the device); raises
        CelloError with CELLO_ENONFINITE if a reduction saw a bad state."""
        w = ctypes.c_uint32()
        _lib.check(_lib.lib().cello_check(self.handle, ctypes.byref(w)), "cello_check")
        return w.value

    # ------------------------------------------------- sharded step, one rank
    def halo_pack(self, U, leaf_ids, buf=None, stream=None):
        """Interiors of the listed leaves into a flat device buffer
        [k, fields, n^3] (allocated if not given); returns it."""
        self._check_state(U)
        ids = np.ascontiguousarray(np.asarray(leaf_ids, dtype=np.int32))
        if buf is None:
            buf = torch.empty(len(ids), self.nf, self.desc.n ** 3, dtype=U.dtype, device=U.device)
        _lib.check(_lib.lib().cello_halo_pack(self.handle, _ptr(U), ids.ctypes.data_as(ctypes.c_void_p), len(ids),
                                              _ptr(buf), _stream(stream)), "cello_halo_pack")
        return buf

    def halo_unpack(self, U, leaf_ids, buf, stream=None):
        self._check_state(U)
        ids = np.ascontiguousarray(np.asarray(leaf_ids, dtype=np.int32))
        if not (buf.is_cuda and buf.dtype == U.dtype and buf.is_contiguous()
                and buf.numel() >= len(ids) * self.nf * self.desc.n ** 3):
            raise CelloError("halo buffer must be a contiguous CUDA tensor of the state's dtype and size")
        _lib.check(_lib.lib().cello_halo_unpack(self.handle, _ptr(U), ids.ctypes.data_as(ctypes.c_void_p), len(ids),
                                                _ptr(buf), _stream(stream)), "cello_halo_unpack")

    def flux_pack(self, faces, buf=None, device="cuda", stream=None):
        """Float64 face fluxes of the listed faces (leaf * 6 + face) into a
        flat device buffer [k, fields, n^2]; returns it."""
        fc = np.ascontiguousarray(np.asarray(faces, dtype=np.int32))
        if buf is None:
            buf = torch.empty(len(fc), self.nf, self.desc.n ** 2, dtype=torch.float64, device=device)
        _lib.check(_lib.lib().cello_flux_pack(self.handle, fc.ctypes.data_as(ctypes.c_void_p), len(fc), _ptr(buf),
                                              _stream(stream)), "cello_flux_pack")
        return buf

    def flux_unpack(self, faces, buf, stream=None):
        fc = np.ascontiguousarray(np.asarray(faces, dtype=np.int32))
        if not (buf.is_cuda and buf.dtype == torch.float64 and buf.is_contiguous()
                and buf.numel() >= len(fc) * self.nf * self.desc.n ** 2):
            raise CelloError("flux buffer must be a contiguous float64 CUDA tensor of the listed size")
        _lib.check(_lib.lib().cello_flux_unpack(self.handle, fc.ctypes.data_as(ctypes.c_void_p), len(fc), _ptr(buf),
                                                _stream(stream)), "cello_flux_unpack")

    def hydro_step_part(self, U, dt, cycle, leaf0, nleaf, part, stream=None):
        self._check_state(U)
        _lib.check(_lib.lib().cello_hydro_step_part(self.handle, _ptr(U), _ptr(dt), int(cycle), int(leaf0), int(nleaf),
                                                    int(part), _stream(stream)), "cello_hydro_step_part")

    def reduce_part(self, U, leaf0, nleaf, out=None, stream=None):
        """[CFL minimum before the factor cfl, five totals] of the leaf range."""
        self._check_state(U)
        if out is None:
            out = torch.empty(6, dtype=torch.float64, device=U.device)
        _lib.check(_lib.lib().cello_reduce_part(self.handle, _ptr(U), int(leaf0), int(nleaf), _ptr(out),
                                                _stream(stream)), "cello_reduce_part")
        return out

    def set_sweep_variant(self, variant: int):
        _lib.check(_lib.lib().cello_set_sweep_variant(self.handle, int(variant)), "cello_set_sweep_variant")

    def autotune(self, U, stream=None):
        """Pick the fastest sweep variant of each axis for this mesh (U is not
        changed).  Returns (chosen variants [x, y, z], best milliseconds of
        each variant as [[x, y, z], ...])."""
        self._check_state(U)
        v = (ctypes.c_int * 3)()
        ms = (ctypes.c_float * 192)()
        _lib.check(_lib.lib().cello_autotune(self.handle, _ptr(U), ctypes.cast(v, ctypes.c_void_p),
                                             ctypes.cast(ms, ctypes.c_void_p), 192, _stream(stream)),
                   "cello_autotune")
        t = [ms[3 * i:3 * i + 3] for i in range(64)]
        return list(v), [list(x) for x in t if any(x)]

    def set_sweep_variants(self, variants):
        """One sweep variant per axis (x, y, z)."""
        arr = (ctypes.c_int * 3)(*[int(x) for x in variants])
        _lib.check(_lib.lib().cello_set_sweep_variants(self.handle, ctypes.cast(arr, ctypes.c_void_p)),
                   "cello_set_sweep_variants")

    def set_exec(self, mode: int):
        _lib.check(_lib.lib().cello_set_exec(self.handle, int(mode)), "cello_set_exec")
