"""Thin ctypes binding of libsph_gb300.so (include/sph.h), same names.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. Tensors are PyTorch CUDA tensors (PyTorch is used for device memory
and streams); their data pointers and the current CUDA stream are passed
through the C ABI. If the library is missing, loading fails loudly -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsph_gb300.so")

SPH_OK = 0
SPH_ERR_INVALID = 1
SPH_ERR_CUDA = 2
SPH_ERR_NOT_CONVERGED = 3
SPH_ERR_H_TOO_LARGE = 4
SPH_ERR_TIMEOUT = 5
SPH_ERR_OOM = 6
STATUS_NAMES = {0: "SPH_OK", 1: "SPH_ERR_INVALID", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_NOT_CONVERGED",
                4: "SPH_ERR_H_TOO_LARGE", 5: "SPH_ERR_TIMEOUT", 6: "SPH_ERR_OOM"}

SPH_FP64 = 0x01
SPH_PLAIN_FP32 = 0x02
SPH_FIXED_H = 0x04
SPH_H_GUESS = 0x08
SPH_TIME_KERNELS = 0x10
SPH_WARP_GROUP = 0x20
SPH_DENSITY_BUFFERED = 0x40
SPH_PER_THREAD_WALK = 0x80
SPH_COOP_WALK = 0x100
SPH_WARP_WALK = 0x200
SPH_NO_LISTS = 0x400
SPH_PARTIAL_LISTS = 0x800

SPH_ST_NOT_CONVERGED = 0x01
SPH_ST_H_TOO_LARGE = 0x02
SPH_ST_TIMEOUT = 0x04
SPH_ST_INVALID = 0x08

EXPORTED = ["sph_default_params", "sph_create", "sph_destroy", "sph_last_error", "sph_build_grid",
            "sph_build_grid_batched", "sph_grid_update", "sph_grid_free", "sph_grid_size", "sph_grid_export",
            "sph_density", "sph_hydro_force", "sph_density_divcurl", "sph_hydro_force_balsara",
            "sph_hydro_force_conduction", "sph_hydro_force_visc", "sph_timebins", "sph_active_from_bins",
            "sph_kick", "sph_drift", "sph_visc_rate", "sph_kick_scalar", "sph_predict_scalar", "sph_gravity", "sph_backward",
            "sph_sync_status", "sph_sort_keys_static"]
SPH_SORT_STATIC_MAX_KEYS = 1 << 20


class sph_params(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("n_target", ctypes.c_double), ("n_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("alpha_visc", ctypes.c_double), ("gamma", ctypes.c_double),
                ("flags", ctypes.c_int), ("group_size", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("walk_radius", ctypes.c_double)]


class sph_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_uint32), ("launches", ctypes.c_uint32),
                ("density_pairs", ctypes.c_uint64), ("force_pairs", ctypes.c_uint64),
                ("density_evals", ctypes.c_uint64), ("pair_tests", ctypes.c_uint64),
                ("groups", ctypes.c_uint64), ("density_kernel_ms", ctypes.c_double),
                ("force_kernel_ms", ctypes.c_double), ("density_launches", ctypes.c_uint32),
                ("force_launches", ctypes.c_uint32), ("grav_nodes", ctypes.c_uint64),
                ("grav_pairs", ctypes.c_uint64), ("list_force", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class sph_gravity_params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("theta", ctypes.c_double), ("r_split", ctypes.c_double),
                ("r_cut", ctypes.c_double), ("h_soft", ctypes.c_double)]


class SPHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load the shared library (build it first with paper_2003_10850_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libsph_gb300.so not found at {p}: run __graft_entry__.build() "
                           "(the CUDA library is required; there is no fallback)")
    L = ctypes.CDLL(p)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    L.sph_default_params.argtypes = [ctypes.POINTER(sph_params)]
    L.sph_default_params.restype = None
    L.sph_create.argtypes = [PP, i32]
    L.sph_create.restype = i32
    L.sph_destroy.argtypes = [P]
    L.sph_destroy.restype = None
    L.sph_last_error.argtypes = [P]
    L.sph_last_error.restype = ctypes.c_char_p
    L.sph_build_grid.argtypes = [P, P, i32, P, i64, ctypes.POINTER(sph_params), P, PP]
    L.sph_build_grid.restype = i32
    L.sph_build_grid_batched.argtypes = [P, P, i32, P, P, P, i32, ctypes.POINTER(sph_params), P, PP]
    L.sph_build_grid_batched.restype = i32
    L.sph_grid_update.argtypes = [P, P, P, i32, P, P]
    L.sph_grid_update.restype = i32
    L.sph_grid_free.argtypes = [P]
    L.sph_grid_free.restype = None
    L.sph_grid_size.argtypes = [P]
    L.sph_grid_size.restype = i64
    L.sph_grid_export.argtypes = [P, P, P, P, P]
    L.sph_grid_export.restype = i32
    L.sph_density.argtypes = [P, P, P, P, i64, P, P, P, P, P, ctypes.POINTER(sph_params), P]
    L.sph_density.restype = i32
    L.sph_hydro_force.argtypes = [P, P, P, P, P, P, P, P, i64, P, P, P, P, ctypes.POINTER(sph_params), P]
    L.sph_hydro_force.restype = i32
    L.sph_density_divcurl.argtypes = [P, P, P, P, i64, P, P, P, P, P, P, P, P, ctypes.POINTER(sph_params), P]
    L.sph_density_divcurl.restype = i32
    L.sph_hydro_force_balsara.argtypes = [P, P, P, P, P, P, P, P, P, P, i64, P, P, P, P,
                                          ctypes.POINTER(sph_params), P]
    L.sph_hydro_force_balsara.restype = i32
    L.sph_hydro_force_conduction.argtypes = [P, P, P, P, P, P, P, P, P, P, P, i64, P, P, P, P, P,
                                             ctypes.POINTER(sph_params), P]
    L.sph_hydro_force_conduction.restype = i32
    L.sph_hydro_force_visc.argtypes = [P, P, P, P, P, P, P, P, P, P, P, i64, P, P, P, P,
                                       ctypes.POINTER(sph_params), P]
    L.sph_hydro_force_visc.restype = i32
    L.sph_visc_rate.argtypes = [P, P, i64, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, P, P]
    L.sph_visc_rate.restype = i32
    L.sph_kick_scalar.argtypes = [P, P, i64, P, P, i32, P, P, P, P]
    L.sph_kick_scalar.restype = i32
    L.sph_predict_scalar.argtypes = [P, i64, ctypes.c_double, P, P, P]
    L.sph_predict_scalar.restype = i32
    L.sph_gravity.argtypes = [P, P, P, i64, ctypes.POINTER(sph_gravity_params), P, P, P, P]
    L.sph_gravity.restype = i32
    L.sph_timebins.argtypes = [P, P, P, P, i64, i64, i64, ctypes.c_double, ctypes.c_double, i32, P, P]
    L.sph_timebins.restype = i32
    L.sph_active_from_bins.argtypes = [P, P, P, i64, i32, P, P, P]
    L.sph_active_from_bins.restype = i32
    L.sph_kick.argtypes = [P, P, i64, P, P, i32, P, P, P, P, P, P, P]
    L.sph_kick.restype = i32
    L.sph_drift.argtypes = [P, P, P, i64, ctypes.c_double, ctypes.c_double, P, P, P, P, P]
    L.sph_drift.restype = i32
    L.sph_backward.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P, ctypes.POINTER(sph_params), P]
    L.sph_backward.restype = i32
    L.sph_sort_keys_static.argtypes = [P, i64, P, P, P]
    L.sph_sort_keys_static.restype = i32
    L.sph_sync_status.argtypes = [P, P, ctypes.POINTER(sph_stats)]
    L.sph_sync_status.restype = i32
    _lib = L
    return L


def default_params(**kw) -> sph_params:
    p = sph_params()
    load().sph_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p
