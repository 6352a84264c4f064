"""ctypes access to the oracle's plain-C direct sums (pairsum.c).

Test infrastructure only.  `build()` compiles pairsum.c with gcc (-O2, OpenMP,
no architecture-specific flags, so it builds the same on x86-64 and Arm).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pairsum.c")
_LIB = os.path.join(_HERE, "_pairsum.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_stokeslet.argtypes = [I64, P, P, I64, P, P, P, ctypes.c_double, P]
        lib.oracle_stresslet.argtypes = [I64, P, I64, P, P, P, P, P]
        lib.oracle_surface_self.argtypes = [I64, P, P, P, P, P]
        lib.oracle_surface_diag.argtypes = [I64, P, P, P, P]
        lib.oracle_body_self.argtypes = [I64, P, P, P, P, P]
        lib.oracle_body_diag.argtypes = [I64, P, P, P, P]
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


def threads() -> int:
    return int(_load().oracle_threads())


def stokeslet(tgt, src, wf, mu=1.0, tgt_fiber=None, src_fiber=None) -> np.ndarray:
    """u_i = sum_j G(x_i - y_j) wf_j, skipping same-fiber pairs when ids are
    given (Eqs. oseen, complementary-uf)."""
    tgt, src, wf = _f64(tgt), _f64(src), _f64(wf)
    tf, sf = _i32(tgt_fiber), _i32(src_fiber)
    out = np.zeros((tgt.shape[0], 3))
    _load().oracle_stokeslet(tgt.shape[0], _p(tgt), _p(tf), src.shape[0], _p(src), _p(sf),
                             _p(wf), float(mu), _p(out))
    return out


def stresslet(tgt, src, normal, w, q) -> np.ndarray:
    """u_i = sum_j w_j T(x_i - y_j):(q_j n_j) at off-surface targets (Eqs. stresslet, double-layer)."""
    tgt, src, normal, w, q = map(_f64, (tgt, src, normal, w, q))
    out = np.zeros((tgt.shape[0], 3))
    _load().oracle_stresslet(tgt.shape[0], _p(tgt), src.shape[0], _p(src), _p(normal), _p(w),
                             _p(q), _p(out))
    return out


def surface_self(y, normal, w, q) -> np.ndarray:
    """q/2 + T_pv[q] + N[q] on the surface nodes (fluid-side limit), by singularity
    subtraction (Eq. main-cortex-density, Sec. 3.1.2)."""
    y, normal, w, q = map(_f64, (y, normal, w, q))
    out = np.zeros((y.shape[0], 3))
    _load().oracle_surface_self(y.shape[0], _p(y), _p(normal), _p(w), _p(q), _p(out))
    return out


def surface_diag(y, normal, w) -> np.ndarray:
    """Diagonal entries of surface_self as a [n, 3] array (Eq. prec)."""
    y, normal, w = map(_f64, (y, normal, w))
    out = np.zeros((y.shape[0], 3))
    _load().oracle_surface_diag(y.shape[0], _p(y), _p(normal), _p(w), _p(out))
    return out


def body_self(y, normal, w, q) -> np.ndarray:
    """-q/2 + T_pv[q] on a rigid body's surface nodes (fluid outside), by
    singularity subtraction (Eq. main-nsb-second-kind, Sec. 3.1.2)."""
    y, normal, w, q = map(_f64, (y, normal, w, q))
    out = np.zeros((y.shape[0], 3))
    _load().oracle_body_self(y.shape[0], _p(y), _p(normal), _p(w), _p(q), _p(out))
    return out


def body_diag(y, normal, w) -> np.ndarray:
    """Diagonal entries of body_self as a [n, 3] array (Eq. prec)."""
    y, normal, w = map(_f64, (y, normal, w))
    out = np.zeros((y.shape[0], 3))
    _load().oracle_body_diag(y.shape[0], _p(y), _p(normal), _p(w), _p(out))
    return out
