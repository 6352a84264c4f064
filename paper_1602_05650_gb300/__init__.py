"""GB300-native implicit step of nonlocal slender-body fibers in Stokes flow.

Thin Python binding of libfibersolve.so (C ABI in include/fibersolve.h).
Every function has the C entry point's name and only marshals arguments:
device arrays are torch CUDA tensors (float64 / int32, contiguous), host
arrays are numpy arrays.  All arithmetic runs in the library's CUDA kernels;
if the library is missing, calls raise ImportError (no CPU fallback).
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _native
from ._native import (FS_FP64, FS_MIXED, FS_SUM_FF, FS_SUM_FP32, FS_SUM_FP32_PLAIN, FS_SUM_FP64,  # noqa: F401
                      fs_boundary, fs_options, fs_step_info)

__all__ = ["fs_options_default", "fs_create", "fs_create_batch", "fs_batch_info", "fs_destroy", "fs_set_state", "fs_get_state",
           "fs_stokeslet_apply", "fs_stresslet_apply", "fs_surface_apply", "fs_build_precond",
           "fs_step", "fs_sizes", "fs_last_error", "fs_kernel_stats", "fs_kernel_launches",
           "fs_probe_fma", "fs_estimate_bytes", "fs_device_bytes", "fs_server_create", "fs_submit",
           "fs_poll", "fs_server_wait", "fs_server_stats", "fs_server_batches", "fs_server_destroy", "Server", "fs_get_self_block", "fs_get_block_lu", "fs_get_tuned_shapes",
           "FsError",
           "fs_set_growth", "fs_get_lengths", "fs_get_unknowns", "fs_dynamic_instability",
           "FS_FP64", "FS_MIXED",
           "FS_SUM_FP32", "FS_SUM_FP64", "FS_SUM_FF", "FS_SUM_FP32_PLAIN"]


class FsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, message, _status_name(status)))


def _status_name(s: int) -> str:
    return _native.load().fs_status_str(int(s)).decode()


def fs_last_error() -> str:
    return _native.load().fs_last_error().decode()


def _check(st: int, where: str):
    if st != 0:
        raise FsError(st, where, fs_last_error())


def _dev_ptr(t, dtype_name: str, name: str):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    want = {"f64": torch.float64, "i32": torch.int32}[dtype_name]
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != want or not t.is_contiguous():
        raise TypeError("%s must be a contiguous %s tensor" % (name, want))
    return ctypes.c_void_p(t.data_ptr())


def _count(t) -> int:
    return int(t.numel()) if hasattr(t, "numel") else int(np.asarray(t).size)


def _need(t, count: int, name: str):
    """The library reads or writes exactly `count` elements of t: refuse any
    other size here (a short array would be overrun)."""
    if t is not None and _count(t) != count:
        raise ValueError("%s has %d elements, %d expected" % (name, _count(t), count))


def _points(t, name: str) -> int:
    """Number of points of an [n, 3] array."""
    shape = tuple(t.shape)
    if len(shape) != 2 or shape[1] != 3:
        raise ValueError("%s must have shape [n, 3] (got %s)" % (name, shape))
    return int(shape[0])


def _checked3(v, name: str):
    a = np.asarray(v, dtype=np.float64).ravel()
    if a.size != 3:
        raise ValueError("%s must have 3 components" % name)
    return a


def _surface_ptrs(obj, what: str):
    """Contiguous float64 nodes [n, 3], normals [n, 3] and weights [n] of a
    boundary or body, sizes checked; returns the arrays and their pointers."""
    nodes, pn = _host_ptr(obj.nodes, np.float64, what + " nodes")
    n = _points(nodes, what + " nodes")
    nrm, pm = _host_ptr(obj.normals, np.float64, what + " normals")
    w, pw = _host_ptr(obj.weights, np.float64, what + " weights")
    _need(nrm, 3 * n, what + " normals")
    _need(w, n, what + " weights")
    return (nodes, nrm, w), (pn, pm, pw), n


def _host_ptr(a, dtype, name: str):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


class Handle:
    """Owns an fs_ctx*; destroyed by fs_destroy (or when collected)."""

    def __init__(self, ptr: ctypes.c_void_p, n_points: int, n_unknowns: int, n_fibers: int):
        self.ptr = ptr
        self.n_points = n_points
        self.n_unknowns = n_unknowns
        self.n_fibers = n_fibers

    def __del__(self):
        try:
            fs_destroy(self)
        except Exception:
            pass


def fs_options_default() -> fs_options:
    o = fs_options()
    _check(_native.load().fs_options_default(ctypes.byref(o)), "fs_options_default")
    return o


def fs_create(points_per_fiber, mu: float, eps: float, E: float, dt: float, boundary=None,
              options: Optional[fs_options] = None, stream=None) -> Handle:
    """points_per_fiber: host int array; boundary: object with R, nodes, normals,
    weights (numpy) or None; stream: torch.cuda.Stream, raw cudaStream_t or None."""
    lib = _native.load()
    ppf, ppf_p = _host_ptr(np.asarray(points_per_fiber), np.int32, "points_per_fiber")
    M = 0 if ppf is None else int(ppf.shape[0])
    b = None
    keep = []
    if boundary is not None:
        arrs, (pn, pm, pw), n = _surface_ptrs(boundary, "boundary")
        keep += list(arrs)
        b = fs_boundary(float(boundary.R), n, pn, pm, pw)
    st = None
    if stream is not None:
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    out = ctypes.c_void_p()
    _check(lib.fs_create(ctypes.byref(out), M, ppf_p, float(mu), float(eps), float(E), float(dt),
                         ctypes.byref(b) if b is not None else None,
                         ctypes.byref(options) if options is not None else None, st), "fs_create")
    npts, nunk = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.fs_sizes(out, ctypes.byref(npts), ctypes.byref(nunk)), "fs_sizes")
    return Handle(out, npts.value, nunk.value, M)


FS_END_FREE, FS_END_CLAMPED, FS_END_HINGED = 0, 1, 2


def fs_create_with_body(points_per_fiber, minus_end, mu: float, eps: float, E: float, dt: float, body,
                        boundary=None, options: Optional[fs_options] = None, stream=None) -> Handle:
    """A context with a rigid body (object with centre, radius, nodes,
    normals, weights, force, torque) and per-fiber minus-end conditions
    (FS_END_*; None = all free)."""
    lib = _native.load()
    ppf, ppf_p = _host_ptr(np.asarray(points_per_fiber), np.int32, "points_per_fiber")
    M = 0 if ppf is None else int(ppf.shape[0])
    keep = []
    me_p = None
    if minus_end is not None:
        me, me_p = _host_ptr(np.asarray(minus_end), np.int32, "minus_end")
        _need(me, M, "minus_end")
        keep.append(me)
    b = None
    if boundary is not None:
        arrs, (pn, pm, pw), n = _surface_ptrs(boundary, "boundary")
        keep += list(arrs)
        b = fs_boundary(float(boundary.R), n, pn, pm, pw)
    arrs, (bpn, bpm, bpw), nb = _surface_ptrs(body, "body")
    keep += list(arrs)
    D3 = ctypes.c_double * 3
    vec3 = lambda v, name: D3(*[float(x) for x in _checked3(v, name)])
    bd = _native.fs_body(vec3(body.centre, "body centre"), float(body.radius), nb, bpn, bpm, bpw,
                         vec3(body.force, "body force"), vec3(body.torque, "body torque"))
    st = None
    if stream is not None:
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    out = ctypes.c_void_p()
    _check(lib.fs_create_with_body(ctypes.byref(out), M, ppf_p, me_p, float(mu), float(eps), float(E), float(dt),
                                   ctypes.byref(b) if b is not None else None, ctypes.byref(bd),
                                   ctypes.byref(options) if options is not None else None, st),
           "fs_create_with_body")
    npts, nunk = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.fs_sizes(out, ctypes.byref(npts), ctypes.byref(nunk)), "fs_sizes")
    return Handle(out, npts.value, nunk.value, M)


def fs_get_body(h: Handle):
    """(centre, U, Omega) of the body, numpy arrays of 3."""
    c, U, Om = (np.zeros(3) for _ in range(3))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(_native.load().fs_get_body(h.ptr, p(c), p(U), p(Om)), "fs_get_body")
    return c, U, Om


def fs_set_body_load(h: Handle, force, torque):
    f = np.ascontiguousarray(force, dtype=np.float64)
    t = np.ascontiguousarray(torque, dtype=np.float64)
    if f.shape != (3,) or t.shape != (3,):
        raise ValueError("force and torque must have 3 components")
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(_native.load().fs_set_body_load(h.ptr, p(f), p(t)), "fs_set_body_load")


def fs_create_batch(fibers_per_system, points_per_fiber, mu: float, eps: float, E: float, dt: float,
                    options: Optional[fs_options] = None, stream=None) -> Handle:
    """Independent free-space systems in one context (see include/fibersolve.h)."""
    lib = _native.load()
    fps, fps_p = _host_ptr(np.asarray(fibers_per_system), np.int32, "fibers_per_system")
    ppf, ppf_p = _host_ptr(np.asarray(points_per_fiber), np.int32, "points_per_fiber")
    _need(ppf, int(fps.astype(np.int64).sum()), "points_per_fiber")   # one entry per fiber of all systems
    st = None
    if stream is not None:
        st = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    out = ctypes.c_void_p()
    _check(lib.fs_create_batch(ctypes.byref(out), int(fps.shape[0]), fps_p, ppf_p, float(mu), float(eps),
                               float(E), float(dt), ctypes.byref(options) if options is not None else None,
                               st), "fs_create_batch")
    npts, nunk = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.fs_sizes(out, ctypes.byref(npts), ctypes.byref(nunk)), "fs_sizes")
    h = Handle(out, npts.value, nunk.value, int(ppf.shape[0]))
    h.n_systems = int(fps.shape[0])
    return h


def fs_batch_info(h: Handle):
    """Per-system iterations, outer steps, residual estimate, converged flag of the last step."""
    S = getattr(h, "n_systems", 1)
    it = np.zeros(S, np.int32)
    ou = np.zeros(S, np.int32)
    rs = np.zeros(S, np.float64)
    cv = np.zeros(S, np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(_native.load().fs_batch_info(h.ptr, p(it), p(ou), p(rs), p(cv)), "fs_batch_info")
    return {"iters": it, "outer": ou, "resid": rs, "converged": cv}


def fs_destroy(h: Handle):
    if h.ptr is not None and h.ptr.value:
        _native.load().fs_destroy(h.ptr)
    h.ptr = None


def fs_sizes(h: Handle):
    return h.n_points, h.n_unknowns


def fs_set_state(h: Handle, X, lengths, f_ext=None):
    """X [N_tot,3], lengths [M], f_ext [N_tot,3]: all CUDA tensors or all numpy arrays."""
    lib = _native.load()
    _need(X, 3 * h.n_points, "X")
    _need(lengths, h.n_fibers, "lengths")
    _need(f_ext, 3 * h.n_points, "f_ext")
    if hasattr(X, "is_cuda") and X.is_cuda:
        _check(lib.fs_set_state(h.ptr, _dev_ptr(X, "f64", "X"), _dev_ptr(lengths, "f64", "lengths"),
                                _dev_ptr(f_ext, "f64", "f_ext"), 1), "fs_set_state")
    else:
        xa, xp = _host_ptr(X, np.float64, "X")
        la, lp = _host_ptr(lengths, np.float64, "lengths")
        fa, fp = _host_ptr(f_ext, np.float64, "f_ext")
        _check(lib.fs_set_state(h.ptr, xp, lp, fp, 0), "fs_set_state")


def fs_get_state(h: Handle, X=None, T=None, V=None):
    """Fill the given output arrays (CUDA tensors or numpy arrays, same kind)."""
    lib = _native.load()
    _need(X, 3 * h.n_points, "X")
    _need(T, h.n_points, "T")
    _need(V, 3 * h.n_points, "V")
    arrs = [a for a in (X, T, V) if a is not None]
    if arrs and hasattr(arrs[0], "is_cuda") and arrs[0].is_cuda:
        _check(lib.fs_get_state(h.ptr, _dev_ptr(X, "f64", "X"), _dev_ptr(T, "f64", "T"),
                                _dev_ptr(V, "f64", "V"), 1), "fs_get_state")
    else:
        for a in arrs:
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
                raise TypeError("host outputs must be C-contiguous float64 numpy arrays")
        p = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
        _check(lib.fs_get_state(h.ptr, p(X), p(T), p(V), 0), "fs_get_state")


def _check_pair_args(src_xyz, src_wf, tgt_xyz, out, src_fiber, tgt_fiber):
    ns, nt = _points(src_xyz, "src_xyz"), _points(tgt_xyz, "tgt_xyz")
    _need(src_wf, 3 * ns, "src_wf")
    _need(out, 3 * nt, "out")
    _need(src_fiber, ns, "src_fiber")
    _need(tgt_fiber, nt, "tgt_fiber")


def fs_stokeslet_apply(h: Handle, src_xyz, src_wf, tgt_xyz, out, src_fiber=None, tgt_fiber=None,
                       sum_precision: int = FS_SUM_FP32):
    lib = _native.load()
    _check_pair_args(src_xyz, src_wf, tgt_xyz, out, src_fiber, tgt_fiber)
    _check(lib.fs_stokeslet_apply(h.ptr, _dev_ptr(src_xyz, "f64", "src_xyz"),
                                  _dev_ptr(src_wf, "f64", "src_wf"), int(src_xyz.shape[0]),
                                  _dev_ptr(src_fiber, "i32", "src_fiber"),
                                  _dev_ptr(tgt_xyz, "f64", "tgt_xyz"),
                                  _dev_ptr(tgt_fiber, "i32", "tgt_fiber"), int(tgt_xyz.shape[0]),
                                  _dev_ptr(out, "f64", "out"), int(sum_precision)),
           "fs_stokeslet_apply")


def fs_stokeslet_apply_tree(h: Handle, src_xyz, src_wf, tgt_xyz, out, src_fiber=None, tgt_fiber=None,
                            order: int = 8, theta: float = 0.5):
    """Treecode approximation of fs_stokeslet_apply (device tensors)."""
    lib = _native.load()
    _check_pair_args(src_xyz, src_wf, tgt_xyz, out, src_fiber, tgt_fiber)
    _check(lib.fs_stokeslet_apply_tree(h.ptr, _dev_ptr(src_xyz, "f64", "src_xyz"),
                                       _dev_ptr(src_wf, "f64", "src_wf"), int(src_xyz.shape[0]),
                                       _dev_ptr(src_fiber, "i32", "src_fiber"),
                                       _dev_ptr(tgt_xyz, "f64", "tgt_xyz"),
                                       _dev_ptr(tgt_fiber, "i32", "tgt_fiber"), int(tgt_xyz.shape[0]),
                                       _dev_ptr(out, "f64", "out"), int(order), float(theta)),
           "fs_stokeslet_apply_tree")


def fs_stresslet_apply(h: Handle, src_xyz, src_nrm, src_w, src_q, tgt_xyz, out,
                       sum_precision: int = FS_SUM_FP32):
    lib = _native.load()
    ns, nt = _points(src_xyz, "src_xyz"), _points(tgt_xyz, "tgt_xyz")
    _need(src_nrm, 3 * ns, "src_nrm")
    _need(src_w, ns, "src_w")
    _need(src_q, 3 * ns, "src_q")
    _need(out, 3 * nt, "out")
    _check(lib.fs_stresslet_apply(h.ptr, _dev_ptr(src_xyz, "f64", "src_xyz"),
                                  _dev_ptr(src_nrm, "f64", "src_nrm"), _dev_ptr(src_w, "f64", "src_w"),
                                  _dev_ptr(src_q, "f64", "src_q"), int(src_xyz.shape[0]),
                                  _dev_ptr(tgt_xyz, "f64", "tgt_xyz"), int(tgt_xyz.shape[0]),
                                  _dev_ptr(out, "f64", "out"), int(sum_precision)),
           "fs_stresslet_apply")


def fs_surface_apply(h: Handle, q, out, sum_precision: int = FS_SUM_FP64):
    # every unknown after the fibers' 4 per node: densities, then the body's U, Omega
    n_surf = h.n_unknowns - 4 * h.n_points
    _need(q, n_surf, "q")
    _need(out, n_surf, "out")
    _check(_native.load().fs_surface_apply(h.ptr, _dev_ptr(q, "f64", "q"), _dev_ptr(out, "f64", "out"),
                                           int(sum_precision)), "fs_surface_apply")


def fs_build_precond(h: Handle):
    _check(_native.load().fs_build_precond(h.ptr), "fs_build_precond")


def fs_step(h: Handle, info: bool = True) -> Optional[fs_step_info]:
    """One implicit step; returns the step info (synchronising) when info=True.
    Raises FsError (status FS_ENOTCONV etc.) on failure."""
    inf = fs_step_info()
    _check(_native.load().fs_step(h.ptr, ctypes.byref(inf) if info else None), "fs_step")
    return inf if info else None


def fs_kernel_stats(h: Handle, reset: bool = False):
    """[(launches, total_ms, pairs)] per direct-sum kernel class (see fs_kernel_class)."""
    arr = (_native.fs_kernel_stat * _native.FS_KS_COUNT)()
    _check(_native.load().fs_kernel_stats(h.ptr, arr, 1 if reset else 0), "fs_kernel_stats")
    return [(a.launches, a.total_ms, a.pairs) for a in arr]


def fs_kernel_launches() -> int:
    return int(_native.load().fs_kernel_launches())


def fs_probe_fma(precision: int) -> float:
    """Measured FMA throughput (flop/s) of the FP64 (0) or FP32 (1) pipe."""
    v = ctypes.c_double()
    _check(_native.load().fs_probe_fma(int(precision), ctypes.byref(v)), "fs_probe_fma")
    return v.value


def fs_estimate_bytes(points_per_fiber, n_surface_nodes: int = 0, options: Optional[fs_options] = None) -> int:
    """Device bytes a context for these fibers (and boundary size) allocates; 0 if invalid."""
    ppf, ppf_p = _host_ptr(np.asarray(points_per_fiber), np.int32, "points_per_fiber")
    return int(_native.load().fs_estimate_bytes(int(ppf.shape[0]), ppf_p, int(n_surface_nodes),
                                                ctypes.byref(options) if options is not None else None))


def fs_device_bytes(h: Handle) -> int:
    v = ctypes.c_size_t()
    _check(_native.load().fs_device_bytes(h.ptr, ctypes.byref(v)), "fs_device_bytes")
    return int(v.value)


class Server:
    """Owns an fs_server*; keeps each pending request's host arrays alive until
    its ticket completes."""

    def __init__(self, ptr: ctypes.c_void_p):
        self.ptr = ptr
        self.pending = {}

    def __del__(self):
        try:
            fs_server_destroy(self)
        except Exception:
            pass


def fs_server_create(hbm_budget_bytes: int, max_slots: int = 4, device: int = 0) -> Server:
    out = ctypes.c_void_p()
    _check(_native.load().fs_server_create(ctypes.byref(out), int(hbm_budget_bytes), int(max_slots), int(device)),
           "fs_server_create")
    return Server(out)


def fs_submit(sv: Server, points_per_fiber, X, lengths, mu: float, eps: float, E: float, dt: float,
              f_ext=None, boundary=None, prec: int = FS_MIXED, tol: float = 0.0) -> int:
    """Queue one step request (host numpy inputs).  Returns the ticket; the
    outputs (X, V, T numpy arrays) are returned by fs_poll / fs_server_wait."""
    ppf, ppf_p = _host_ptr(np.asarray(points_per_fiber), np.int32, "points_per_fiber")
    n_tot = int(ppf.sum())
    _need(X, 3 * n_tot, "X")
    _need(lengths, int(ppf.shape[0]), "lengths")
    _need(f_ext, 3 * n_tot, "f_ext")
    xa, xp = _host_ptr(X, np.float64, "X")
    la, lp = _host_ptr(lengths, np.float64, "lengths")
    fa, fp = _host_ptr(f_ext, np.float64, "f_ext")
    outs = (np.zeros((n_tot, 3)), np.zeros((n_tot, 3)), np.zeros(n_tot))
    keep = [ppf, xa, la, fa, outs]
    bptr = None
    if boundary is not None:
        arrs, (pn, pm, pw), n = _surface_ptrs(boundary, "boundary")
        b = fs_boundary(float(boundary.R), n, pn, pm, pw)
        keep += list(arrs) + [b]
        bptr = ctypes.pointer(b)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rq = _native.fs_request(int(ppf.shape[0]), ppf_p, xp, lp, fp, bptr, float(mu), float(eps), float(E),
                            float(dt), int(prec), float(tol), p(outs[0]), p(outs[1]), p(outs[2]))
    t = ctypes.c_uint64()
    _check(_native.load().fs_submit(sv.ptr, ctypes.byref(rq), ctypes.byref(t)), "fs_submit")
    sv.pending[t.value] = keep
    return int(t.value)


def _complete(sv: Server, ticket: int, st: int, inf, where: str):
    keep = sv.pending.pop(ticket, None)
    _check(st, where)
    X, V, T = keep[4]
    return {"X": X, "V": V, "T": T, "info": inf}


def fs_poll(sv: Server, ticket: int):
    """None while the request is queued or running, else its result dict
    (X, V, T, info); raises FsError if the request failed."""
    inf = fs_step_info()
    st = _native.load().fs_poll(sv.ptr, int(ticket), ctypes.byref(inf))
    if st == _native.FS_EAGAIN:
        return None
    return _complete(sv, int(ticket), st, inf, "fs_poll")


def fs_server_wait(sv: Server, ticket: int, timeout_s: float = 600.0):
    inf = fs_step_info()
    st = _native.load().fs_server_wait(sv.ptr, int(ticket), ctypes.byref(inf), float(timeout_s))
    if st == _native.FS_ETIMEOUT:
        raise FsError(st, "fs_server_wait", fs_last_error())
    return _complete(sv, int(ticket), st, inf, "fs_server_wait")


def fs_server_stats(sv: Server):
    pe, ru, co = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    by = ctypes.c_size_t()
    _check(_native.load().fs_server_stats(sv.ptr, ctypes.byref(pe), ctypes.byref(ru), ctypes.byref(by),
                                          ctypes.byref(co)), "fs_server_stats")
    return {"pending": pe.value, "running": ru.value, "bytes_in_use": int(by.value), "completed": co.value}


def fs_get_self_block(h: Handle, fiber: int, n_points: int):
    """The assembled self block of one fiber as a (4N, 4N) numpy array."""
    n = 4 * int(n_points)
    out = np.zeros(n * n)
    _check(_native.load().fs_get_self_block(h.ptr, int(fiber), out.ctypes.data_as(ctypes.c_void_p)),
           "fs_get_self_block")
    return out.reshape(n, n).T   # column-major storage


def fs_get_block_lu(h: Handle, fiber: int, n_points: int):
    """The LU factors of one fiber's self block: (LU, piv) with LU the (4N, 4N)
    array holding L below the diagonal (unit diagonal implied) and U on and
    above it, and P B = L U where row i of P B is row piv[i] of B."""
    n = 4 * int(n_points)
    lu = np.zeros(n * n)
    piv = np.zeros(n, dtype=np.int32)
    _check(_native.load().fs_get_block_lu(h.ptr, int(fiber), lu.ctypes.data_as(ctypes.c_void_p),
                                          piv.ctypes.data_as(ctypes.c_void_p)), "fs_get_block_lu")
    return lu.reshape(n, n).T, piv


def fs_get_tuned_shapes(h: Handle):
    """The far field's autotuned launch shapes: {(sum precision, hi/lo): shape
    id 1..3} for the classes tuned so far (fs_options.autotune)."""
    out = np.zeros(8, dtype=np.int32)
    _check(_native.load().fs_get_tuned_shapes(h.ptr, out.ctypes.data_as(ctypes.c_void_p)),
           "fs_get_tuned_shapes")
    return {(p, hl): int(out[2 * p + hl]) for p in range(4) for hl in range(2) if out[2 * p + hl]}


def fs_server_batches(sv: Server) -> int:
    n = ctypes.c_int64()
    _check(_native.load().fs_server_batches(sv.ptr, ctypes.byref(n)), "fs_server_batches")
    return int(n.value)


def fs_server_destroy(sv: Server):
    if sv.ptr is not None and sv.ptr.value:
        _native.load().fs_server_destroy(sv.ptr)
    sv.ptr = None
    sv.pending.clear()


def fs_set_growth(h: Handle, Ldot):
    """Per-fiber plus-end growth rates: a CUDA tensor or a numpy array."""
    lib = _native.load()
    _need(Ldot, h.n_fibers, "Ldot")
    if hasattr(Ldot, "is_cuda") and Ldot.is_cuda:
        _check(lib.fs_set_growth(h.ptr, _dev_ptr(Ldot, "f64", "Ldot"), 1), "fs_set_growth")
    else:
        a, p = _host_ptr(Ldot, np.float64, "Ldot")
        _check(lib.fs_set_growth(h.ptr, p, 0), "fs_set_growth")


def fs_get_lengths(h: Handle, M: int):
    if int(M) != h.n_fibers:
        raise ValueError("the context has %d fibers, not %d" % (h.n_fibers, int(M)))
    out = np.zeros(int(M))
    _check(_native.load().fs_get_lengths(h.ptr, out.ctypes.data_as(ctypes.c_void_p), 0), "fs_get_lengths")
    return out


def fs_dynamic_instability(state, lengths, u, dt: float, v_grow: float, v_shrink: float, f_cat: float,
                           f_res: float, L_min: float, L_max: float = 0.0):
    """One step of the two-state dynamic instability (host, no GPU): returns
    (new_state int32, Ldot) for the given per-fiber uniform random numbers u."""
    st = np.ascontiguousarray(state, dtype=np.int32).copy()
    _need(lengths, st.size, "lengths")
    _need(u, st.size, "u")
    La, Lp = _host_ptr(lengths, np.float64, "lengths")
    ua, up = _host_ptr(u, np.float64, "u")
    Ld = np.zeros(st.shape[0])
    k = _native.fs_kinetics(float(v_grow), float(v_shrink), float(f_cat), float(f_res), float(L_min), float(L_max))
    _check(_native.load().fs_dynamic_instability(int(st.shape[0]), ctypes.byref(k), float(dt), Lp, up,
                                                 st.ctypes.data_as(ctypes.c_void_p),
                                                 Ld.ctypes.data_as(ctypes.c_void_p)), "fs_dynamic_instability")
    return st, Ld


def fs_get_unknowns(h: Handle):
    """The last solve's unknown vector (host numpy array of fs_sizes()[1])."""
    out = np.zeros(int(h.n_unknowns))
    _check(_native.load().fs_get_unknowns(h.ptr, out.ctypes.data_as(ctypes.c_void_p), 0), "fs_get_unknowns")
    return out
