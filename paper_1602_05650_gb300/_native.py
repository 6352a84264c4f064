"""ctypes declarations of the C ABI in include/fibersolve.h (argument
marshalling only; every computation happens in libfibersolve.so).

Loading fails loudly when the library has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfibersolve.so")

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p
P = c_void_p

FS_OK, FS_EINVAL, FS_ENOMEM, FS_ECUDA, FS_ENOTCONV, FS_ENUMERIC, FS_EAGAIN, FS_EBUSY, FS_ETIMEOUT = range(9)
FS_FP64, FS_MIXED = 0, 1
FS_SUM_FP64, FS_SUM_FP32, FS_SUM_FF, FS_SUM_FP32_PLAIN = 0, 1, 2, 3


class fs_boundary(ctypes.Structure):
    _fields_ = [("R", c_double), ("n_nodes", c_int32), ("nodes", P), ("normals", P), ("weights", P)]


class fs_body(ctypes.Structure):
    _fields_ = [("center", c_double * 3), ("radius", c_double), ("n_nodes", c_int32), ("nodes", P),
                ("normals", P), ("weights", P), ("force", c_double * 3), ("torque", c_double * 3)]


class fs_options(ctypes.Structure):
    _fields_ = [("prec", c_int32), ("tol", c_double), ("max_iter", c_int32), ("restart", c_int32),
                ("max_refine", c_int32), ("inner_tol", c_double), ("delta_over_L", c_double),
                ("lsb", c_int32), ("use_graph", c_int32), ("tile_override", c_int32),
                ("profile", c_int32), ("relax", c_int32), ("tree_order", c_int32), ("tree_theta", c_double),
                ("growth_implicit", c_int32), ("tc_blocks", c_int32), ("tc_lu", c_int32),
                ("autotune", c_int32)]


class fs_kernel_stat(ctypes.Structure):
    _fields_ = [("launches", c_int64), ("total_ms", c_double), ("pairs", c_double)]


FS_KS_COUNT = 8


class fs_step_info(ctypes.Structure):
    _fields_ = [("iters", c_int32), ("refine_sweeps", c_int32), ("resid", c_double),
                ("t_ms", c_double * 8), ("pairs", c_int64)]


class fs_request(ctypes.Structure):
    _fields_ = [("n_fibers", c_int32), ("points_per_fiber", P), ("X", P), ("lengths", P), ("f_ext", P),
                ("boundary", ctypes.POINTER(fs_boundary)), ("mu", c_double), ("eps", c_double),
                ("E", c_double), ("dt", c_double), ("prec", c_int32), ("tol", c_double),
                ("out_X", P), ("out_V", P), ("out_T", P)]


class fs_kinetics(ctypes.Structure):
    _fields_ = [("v_grow", c_double), ("v_shrink", c_double), ("f_cat", c_double), ("f_res", c_double),
                ("L_min", c_double), ("L_max", c_double)]


# name -> (restype, argtypes)
SIGNATURES = {
    "fs_options_default": (c_int32, [ctypes.POINTER(fs_options)]),
    "fs_create": (c_int32, [ctypes.POINTER(c_void_p), c_int32, P, c_double, c_double, c_double,
                            c_double, ctypes.POINTER(fs_boundary), ctypes.POINTER(fs_options), P]),
    "fs_destroy": (None, [P]),
    "fs_create_batch": (c_int32, [ctypes.POINTER(c_void_p), c_int32, P, P, c_double, c_double, c_double,
                                  c_double, ctypes.POINTER(fs_options), P]),
    "fs_batch_info": (c_int32, [P, P, P, P, P]),
    "fs_set_state": (c_int32, [P, P, P, P, c_int32]),
    "fs_get_state": (c_int32, [P, P, P, P, c_int32]),
    "fs_stokeslet_apply": (c_int32, [P, P, P, c_int64, P, P, P, c_int64, P, c_int32]),
    "fs_stresslet_apply": (c_int32, [P, P, P, P, P, c_int64, P, c_int64, P, c_int32]),
    "fs_stokeslet_apply_tree": (c_int32, [P, P, P, c_int64, P, P, P, c_int64, P, c_int32, c_double]),
    "fs_stokeslet_apply_noalloc": (c_int32, [P, P, c_int64, P, P, P, c_int64, P, c_double, c_int32, P]),
    "fs_surface_apply": (c_int32, [P, P, P, c_int32]),
    "fs_build_precond": (c_int32, [P]),
    "fs_step": (c_int32, [P, ctypes.POINTER(fs_step_info)]),
    "fs_sizes": (c_int32, [P, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64)]),
    "fs_kernel_stats": (c_int32, [P, ctypes.POINTER(fs_kernel_stat), c_int32]),
    "fs_kernel_launches": (ctypes.c_uint64, []),
    "fs_probe_fma": (c_int32, [c_int32, ctypes.POINTER(c_double)]),
    "fs_set_growth": (c_int32, [P, P, c_int32]),
    "fs_get_lengths": (c_int32, [P, P, c_int32]),
    "fs_get_unknowns": (c_int32, [P, P, c_int32]),
    "fs_create_with_body": (c_int32, [ctypes.POINTER(c_void_p), c_int32, P, P, c_double, c_double, c_double,
                                      c_double, P, P, P, c_void_p]),
    "fs_get_body": (c_int32, [P, P, P, P]),
    "fs_set_body_load": (c_int32, [P, P, P]),
    "fs_dynamic_instability": (c_int32, [c_int32, ctypes.POINTER(fs_kinetics), c_double, P, P, P, P]),
    "fs_estimate_bytes": (ctypes.c_size_t, [c_int32, P, c_int32, ctypes.POINTER(fs_options)]),
    "fs_device_bytes": (c_int32, [P, ctypes.POINTER(ctypes.c_size_t)]),
    "fs_server_create": (c_int32, [ctypes.POINTER(c_void_p), ctypes.c_size_t, c_int32, c_int32]),
    "fs_submit": (c_int32, [P, ctypes.POINTER(fs_request), ctypes.POINTER(ctypes.c_uint64)]),
    "fs_poll": (c_int32, [P, ctypes.c_uint64, ctypes.POINTER(fs_step_info)]),
    "fs_server_wait": (c_int32, [P, ctypes.c_uint64, ctypes.POINTER(fs_step_info), c_double]),
    "fs_server_stats": (c_int32, [P, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                  ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(c_int64)]),
    "fs_server_destroy": (None, [P]),
    "fs_server_batches": (c_int32, [P, ctypes.POINTER(c_int64)]),
    "fs_get_self_block": (c_int32, [P, c_int32, P]),
    "fs_get_block_lu": (c_int32, [P, c_int32, P, P]),
    "fs_get_tuned_shapes": (c_int32, [P, P]),
    "fs_last_error": (ctypes.c_char_p, []),
    "fs_status_str": (ctypes.c_char_p, [c_int32]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libfibersolve.so (built by paper_1602_05650_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfibersolve.so is not built; run paper_1602_05650_gb300.build.build() "
                              "(needs nvcc). There is no CPU fallback.")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(SIGNATURES)
