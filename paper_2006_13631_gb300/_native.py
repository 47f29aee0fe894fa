"""ctypes declarations of the C ABI in include/hlbm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhlbm.so")

HLBM_OK, HLBM_EINVAL, HLBM_ECUDA, HLBM_EUNSTABLE, HLBM_EGEOM, HLBM_ENOMEM, HLBM_EIO = 0, -1, -2, -3, -4, -5, -6
HLBM_ETIMEOUT = -7
HLBM_FAULT_STALL_TILE, HLBM_FAULT_NAN_LATTICE = 1, 2
HLBM_FV_AUTO, HLBM_FV_GLOBAL, HLBM_FV_SMEM, HLBM_FV_TMEM, HLBM_FV_DEEP = 0, 1, 2, 3, 4
HLBM_BC_WALL, HLBM_BC_OUTFLOW, HLBM_BC_PERIODIC = 0, 1, 2
HLBM_F64, HLBM_F32, HLBM_F16, HLBM_BF16 = 0, 1, 2, 3
HLBM_NODE_INTERIOR, HLBM_NODE_OUTER, HLBM_NODE_WALL = 0, 1, 2
HLBM_MOTION_STATIC, HLBM_MOTION_HARMONIC, HLBM_MOTION_UNIFORM, HLBM_MOTION_INDUCED = 0, 1, 2, 3
HLBM_ST_FILL_NOT_LOCATED, HLBM_ST_DONOR_NOT_COMPUTED, HLBM_ST_NONFINITE, HLBM_ST_UNUSED_TO_DISC = 1, 2, 8, 16
HLBM_ST_SYNC_TIMEOUT = 32
PHASES = ("move", "stream", "fv", "force")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


MAX_LEVELS = 4


class hlbm_level_t(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("ox", C.c_int32), ("oy", C.c_int32),
                ("rho_init", _dp), ("ux_init", _dp), ("uy_init", _dp)]


class hlbm_grid_t(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32),
                ("dtype", C.c_int32), ("rho0", C.c_double), ("u0x", C.c_double), ("u0y", C.c_double),
                ("rho_init", _dp), ("ux_init", _dp), ("uy_init", _dp),
                ("n_levels", C.c_int32), ("levels", C.POINTER(hlbm_level_t)),
                ("sponge_rows", C.c_int32), ("sponge_sigma", C.c_double)]


class hlbm_patch_t(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_tris", C.c_int32), ("xy", _dp), ("tri", _ip),
                ("kind", C.POINTER(C.c_int8)), ("lamina_L", C.c_double), ("lamina_T", C.c_double),
                ("x_c", C.c_double), ("y_c", C.c_double), ("delta_f", C.c_double),
                ("n_sub", C.c_int32), ("lumped", C.c_int32), ("outer_fv", C.c_int32), ("fv_kernel", C.c_int32)]


class hlbm_motion_t(C.Structure):
    _fields_ = [("kind", C.c_int32), ("A", C.c_double), ("omega", C.c_double),
                ("vx", C.c_double), ("vy", C.c_double), ("mass", C.c_double), ("stiffness", C.c_double),
                ("damping", C.c_double), ("y0", C.c_double), ("v0", C.c_double)]


class hlbm_info_t(C.Structure):
    _fields_ = [("time", C.c_int64), ("n_struct", C.c_int64), ("n_struct_disc", C.c_int64),
                ("n_nodes", C.c_int32), ("n_tris", C.c_int32), ("nnz", C.c_int32), ("n_outer", C.c_int32),
                ("n_wall_segments", C.c_int32), ("box_w", C.c_int32), ("box_h", C.c_int32),
                ("launches_per_step", C.c_int32), ("dtype", C.c_int32), ("fv_kernel", C.c_int32),
                ("n_tiles", C.c_int32), ("y", C.c_double), ("vy", C.c_double), ("n_levels", C.c_int32),
                ("n_coarse", C.c_int64), ("coarse_updates", C.c_double), ("fv_depth", C.c_int32),
                ("fv_slots", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# every entry point declared in include/hlbm.h: name -> (restype, argtypes)
SIGNATURES = {
    "hlbm_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    "hlbm_create": (C.c_int, [C.POINTER(hlbm_grid_t), C.POINTER(hlbm_patch_t), C.c_double,
                              C.POINTER(hlbm_motion_t), C.c_void_p, C.POINTER(C.c_void_p)]),
    "hlbm_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "hlbm_force": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, _dp, _dp]),
    "hlbm_gamma": (C.c_int, [C.c_void_p, C.c_double, C.c_double, _dp, _dp, _dp]),
    "hlbm_get_fields": (C.c_int, [C.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp]),
    "hlbm_get_level_fields": (C.c_int, [C.c_void_p, C.c_int32, _dp, _dp, _dp]),
    "hlbm_get_class": (C.c_int, [C.c_void_p, C.POINTER(C.c_int8)]),
    "hlbm_get_refill": (C.c_int, [C.c_void_p, _ip, _ip]),
    "hlbm_get_patch_f": (C.c_int, [C.c_void_p, _dp]),
    "hlbm_get_fv": (C.c_int, [C.c_void_p, _ip, _ip, _dp, _dp, _dp]),
    "hlbm_info": (C.c_int, [C.c_void_p, C.POINTER(hlbm_info_t)]),
    "hlbm_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32)]),
    "hlbm_clear_status": (C.c_int, [C.c_void_p]),
    "hlbm_set_fv_depth": (C.c_int, [C.c_void_p, C.c_int32]),
    "hlbm_set_overlap": (C.c_int, [C.c_void_p, C.c_int32]),
    "hlbm_set_overlap_share": (C.c_int, [C.c_void_p, C.c_double]),
    "hlbm_inject_fault": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "hlbm_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "hlbm_profile_read": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64)]),
    "hlbm_fit_static": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_void_p, _dp, _dp,
                                  _dp]),
    "hlbm_sweep_create": (C.c_int, [C.c_int32, C.POINTER(C.c_void_p), C.c_void_p, C.POINTER(C.c_void_p)]),
    "hlbm_sweep_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "hlbm_sweep_tune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "hlbm_sweep_fv_time": (C.c_int, [C.c_void_p, C.c_int64, _dp]),
    "hlbm_sweep_pack": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "hlbm_sweep_last_error": (C.c_char_p, [C.c_void_p]),
    "hlbm_sweep_destroy": (None, [C.c_void_p]),
    "hlbm_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "hlbm_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "hlbm_theta_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_int64, C.c_double,
                                      C.c_double, C.c_double, C.c_void_p, _dp, _dp, _dp]),
    "hlbm_theta_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_int64, C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_int32, C.c_void_p, _dp, _dp, _dp, _dp]),
    "hlbm_last_error": (C.c_char_p, [C.c_void_p]),
    "hlbm_destroy": (None, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run paper_2006_13631_gb300.build.build())")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
