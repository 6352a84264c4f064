"""fs_stokeslet_apply_noalloc: the direct Stokeslet sum for callers that cannot
let the library allocate device memory (its scratch is a fixed array in
device memory).  Called through the C ABI and compared with fs_stokeslet_apply
on the same inputs, twice in a row with different inputs (the shared scratch
keeps the previous call's contents), in every precision, with and without
fiber ids, with separate source and target sets, at the largest size the
header documents, plus the size limit.  Runs last."""
import ctypes

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402
from paper_1602_05650_gb300 import _native  # noqa: E402

# the tolerances of the direct-sum parity tests for each precision
TOL = {fs.FS_SUM_FP32: 1e-6, fs.FS_SUM_FP32_PLAIN: 1e-6, fs.FS_SUM_FP64: 1e-12, fs.FS_SUM_FF: 5e-11}
PRECS = [fs.FS_SUM_FP32, fs.FS_SUM_FP32_PLAIN, fs.FS_SUM_FP64, fs.FS_SUM_FF]


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def dev(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda:0")


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _noalloc(lib, src, w, sid, tgt, tid, mu, prec, stream):
    out = torch.full_like(tgt, float("nan"))
    st = lib.fs_stokeslet_apply_noalloc(_p(src), _p(w), src.shape[0], _p(sid), _p(tgt), _p(tid),
                                        tgt.shape[0], _p(out), mu, prec,
                                        ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, fs.fs_last_error()
    return out


@pytest.mark.parametrize("ids", [True, False])
@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_matches_context_path_twice(prec, ids):
    lib = _native.load()
    mu = 1.7
    h = fs.fs_create([], mu, 1e-3, 1.0, 1e-3)
    stream = torch.cuda.current_stream()
    for seed, (M, N) in enumerate([(40, 32), (23, 24)]):
        s = wl.free_space(M, N, 8.0, seed=seed, curved_amp=0.05)
        X, W = dev(s.X), dev(s.f_ext * 0.05)
        fid = dev(s.fiber_id(), torch.int32) if ids else None
        # without ids every pair counts: targets offset from the sources
        T = X if ids else X + 0.0137
        ref = torch.empty_like(T)
        fs.fs_stokeslet_apply(h, X, W, T, ref, fid, fid, prec)
        out = _noalloc(lib, X, W, fid, T, fid, mu, prec, stream)
        torch.cuda.synchronize()
        assert rel(out, ref) <= TOL[prec]
    fs.fs_destroy(h)


@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_separate_sources_and_targets(prec):
    """n_src != n_tgt, a ragged number of each, no ids."""
    lib = _native.load()
    mu = 0.8
    h = fs.fs_create([], mu, 1e-3, 1.0, 1e-3)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    src = dev(rng.uniform(0.0, 6.0, size=(3001, 3)))
    w = dev(rng.normal(size=(3001, 3)))
    tgt = dev(rng.uniform(0.0, 6.0, size=(517, 3)))
    ref = torch.empty_like(tgt)
    fs.fs_stokeslet_apply(h, src, w, tgt, ref, None, None, prec)
    out = _noalloc(lib, src, w, None, tgt, None, mu, prec, stream)
    torch.cuda.synchronize()
    assert rel(out, ref) <= TOL[prec]
    fs.fs_destroy(h)


@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_at_the_documented_size(prec):
    """65,536 sources and targets with fiber ids (the size the header states
    the fixed scratch admits on GB300) is accepted and matches the context
    path."""
    lib = _native.load()
    s = wl.cfg_cloud_mixed(0)
    mu = s.mu
    h = fs.fs_create([], mu, 1e-3, 1.0, 1e-3)
    stream = torch.cuda.current_stream()
    X, W = dev(s.X), dev(s.f_ext * 0.02)
    fid = dev(s.fiber_id(), torch.int32)
    ref = torch.empty_like(X)
    fs.fs_stokeslet_apply(h, X, W, X, ref, fid, fid, prec)
    out = _noalloc(lib, X, W, fid, X, fid, mu, prec, stream)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)   # same kernels, same launch shape, same order
    fs.fs_destroy(h)


def test_noalloc_rejects_beyond_its_scratch():
    lib = _native.load()
    n = 2_000_000
    st = lib.fs_stokeslet_apply_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), n, None,
                                        ctypes.c_void_p(16), None, n, ctypes.c_void_p(16), 1.0,
                                        fs.FS_SUM_FP32, None)
    assert st == _native.FS_EINVAL
    assert "scratch" in fs.fs_last_error()
