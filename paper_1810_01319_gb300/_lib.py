"""ctypes binding of libcello_gpu.so (include/cello.h).  Argument marshalling
only: every step of the hydro path runs in the library's CUDA kernels.  The
library must be built (paper_1810_01319_gb300.build); nothing falls back to
a CPU implementation."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcello_gpu.so")

PERIODIC, OUTFLOW = 0, 1
EXEC_PLAIN, EXEC_BATCHED, EXEC_GRAPH = 0, 1, 2

STATUS = {0: "CELLO_OK", 1: "CELLO_EINVAL", 2: "CELLO_ENOMEM", 3: "CELLO_ECUDA", 4: "CELLO_ENONFINITE",
          5: "CELLO_ETIMEOUT", 6: "CELLO_EINTERNAL"}


class MeshDesc(ctypes.Structure):
    _fields_ = [("root", ctypes.c_int * 3), ("n", ctypes.c_int), ("ghosts", ctypes.c_int),
                ("max_level", ctypes.c_int), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 3), ("precision", ctypes.c_int), ("gamma", ctypes.c_double),
                ("riemann", ctypes.c_int), ("steepening", ctypes.c_int),
                ("dual_energy", ctypes.c_int)]


class CelloError(RuntimeError):
    pass


_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); must list every entry point of include/cello.h
SIGNATURES = {
    "cello_octree_build": (ctypes.c_int, [ctypes.POINTER(MeshDesc), _vp, _vp, ctypes.POINTER(_vp)]),
    "cello_mesh_free": (None, [_vp]),
    "cello_mesh_from_leaves": (ctypes.c_int, [ctypes.POINTER(MeshDesc), _vp, ctypes.c_int64, ctypes.POINTER(_vp)]),
    "cello_check": (ctypes.c_int, [_vp, _vp]),
    "cello_particles_locate": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp]),
    "cello_poisson_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "cello_particles_push": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp]),
    "cello_hydro_step_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _vp, ctypes.c_int, ctypes.c_double,
                                             _vp, _vp, _vp]),
    "cello_sweep_opcount": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int, _vp]),
    "cello_mesh_info": (ctypes.c_int, [_vp, _i64p, _i64p, _i64p]),
    "cello_mesh_leaves": (ctypes.c_int, [_vp, _vp]),
    "cello_neighbour_table": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "cello_refine_flags": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "cello_ghost_refresh": (ctypes.c_int, [_vp, _vp, _vp]),
    "cello_remap": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "cello_hydro_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, _vp, _vp, _vp]),
    "cello_hydro_step_cfl": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_double, _vp, _vp, _vp]),
    "cello_reduce": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    "cello_reduce_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    "cello_fp32_ffma_rate": (ctypes.c_int, [_vp, _vp, _vp]),
    "cello_halo_pack": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp]),
    "cello_halo_unpack": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp]),
    "cello_flux_pack": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp]),
    "cello_flux_unpack": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp]),
    "cello_hydro_step_part": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int, _vp]),
    "cello_reduce_part": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int64, _vp, _vp]),
    "cello_set_exec": (ctypes.c_int, [_vp, ctypes.c_int]),
    "cello_set_sweep_variant": (ctypes.c_int, [_vp, ctypes.c_int]),
    "cello_set_sweep_variants": (ctypes.c_int, [_vp, _vp]),
    "cello_autotune": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "cello_hydro_adjoint_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "cello_profile_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, _vp, _vp]),
    "cello_last_error": (ctypes.c_char_p, []),
}

_LIB = None


def lib():
    """Load the library (once).  Raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise CelloError(f"{LIB_PATH} is missing: build it with paper_1810_01319_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(status: int, what: str):
    if status != 0:
        msg = lib().cello_last_error().decode()
        raise CelloError(f"{what} failed with {STATUS.get(status, status)}: {msg}")
