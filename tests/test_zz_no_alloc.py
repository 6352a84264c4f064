"""fs_stokeslet_apply_noalloc: the direct Stokeslet sum for callers that cannot
let the library allocate device memory (its scratch is a fixed array in
device memory).  Called through the C ABI and compared with fs_stokeslet_apply
on the same inputs, twice in a row with different inputs (the shared scratch
keeps the previous call's contents), plus the size limit.  Runs last."""
import ctypes

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1602_05650_gb300 as fs  # noqa: E402
from paper_1602_05650_gb300 import _native  # noqa: E402

TOL = {fs.FS_SUM_FP32: 1e-6, fs.FS_SUM_FP64: 1e-12, 2: 5e-11}


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def dev(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda:0")


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("prec", [fs.FS_SUM_FP32, fs.FS_SUM_FP64, 2])
def test_noalloc_matches_context_path_twice(prec):
    lib = _native.load()
    mu = 1.7
    h = fs.fs_create([], mu, 1e-3, 1.0, 1e-3)
    stream = torch.cuda.current_stream()
    for seed, (M, N) in enumerate([(40, 32), (23, 24)]):
        s = wl.free_space(M, N, 8.0, seed=seed, curved_amp=0.05)
        X, W = dev(s.X), dev(s.f_ext * 0.05)
        fid = dev(s.fiber_id(), torch.int32)
        ref = torch.empty_like(X)
        fs.fs_stokeslet_apply(h, X, W, X, ref, fid, fid, prec)
        out = torch.full_like(X, float("nan"))
        st = lib.fs_stokeslet_apply_noalloc(_p(X), _p(W), X.shape[0], _p(fid), _p(X), _p(fid),
                                            X.shape[0], _p(out), mu, prec,
                                            ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, fs.fs_last_error()
        torch.cuda.synchronize()
        assert rel(out, ref) <= TOL[prec]
    fs.fs_destroy(h)


def test_noalloc_rejects_beyond_its_scratch():
    lib = _native.load()
    n = 2_000_000
    st = lib.fs_stokeslet_apply_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), n, None,
                                        ctypes.c_void_p(16), None, n, ctypes.c_void_p(16), 1.0,
                                        fs.FS_SUM_FP32, None)
    assert st == _native.FS_EINVAL
    assert "scratch" in fs.fs_last_error()
