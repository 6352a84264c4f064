"""Host-side logic of the serving front end and of the device-memory estimate
(no GPU: fs_estimate_bytes makes no CUDA call; server entry points validate
their arguments before touching a device)."""
import ctypes

import numpy as np
import pytest

from paper_1602_05650_gb300 import _native, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def est(lib, ppf, ns=0, prec=_native.FS_MIXED, restart=60, tc_blocks=1, tc_lu=1):
    a = np.asarray(ppf, np.int32)
    o = _native.fs_options()
    lib.fs_options_default(ctypes.byref(o))
    o.prec = prec
    o.restart = restart
    o.tc_blocks = tc_blocks
    o.tc_lu = tc_lu
    return lib.fs_estimate_bytes(len(a), a.ctypes.data_as(ctypes.c_void_p), ns, ctypes.byref(o))


def test_estimate_grows_with_the_problem(lib):
    e1 = est(lib, [32] * 100)
    e2 = est(lib, [32] * 200)
    assert 0 < e1 < e2
    # the dense blocks and the block-build scratch (16 + 3 + 12 N^2 doubles
    # per fiber) dominate at N = 64 with the FP64 build and LU
    e64 = est(lib, [64] * 1024, tc_blocks=0, tc_lu=0)
    assert e64 >= 1024 * 31 * 64 * 64 * 8
    assert e64 < 2 * 1024 * 31 * 64 * 64 * 8
    # the tensor-core build adds the digit planes of a chunk of 512 fibers:
    # nine bf16 planes of both operands (256 rows each, 192 inner columns)
    planes = 512 * 9 * (256 + 256) * 192 * 2
    # (the LU's planes fit in them)
    assert planes <= est(lib, [64] * 1024) - e64 < planes + (16 << 20)
    # the tensor-core LU alone: planes for all 1,024 fibers, nine bf16 planes
    # of both operands (256 rows, 32 inner columns) and an exponent per row
    lu = 1024 * 2 * (9 * 256 * 32 * 2 + 256 * 4)
    assert lu <= est(lib, [64] * 1024, tc_blocks=0) - e64 < lu + (16 << 20)
    # beyond 4N = 512 the LU stays on the FP64 pipe and allocates no planes
    assert est(lib, [160] * 8, tc_blocks=0) == est(lib, [160] * 8, tc_blocks=0, tc_lu=0)
    assert est(lib, [128] * 8, tc_blocks=0) > est(lib, [128] * 8, tc_blocks=0, tc_lu=0)
    # mixed precision keeps the outer flexible-GMRES space on top of the inner one
    assert est(lib, [32] * 100, prec=_native.FS_MIXED) > est(lib, [32] * 100, prec=_native.FS_FP64)
    # a longer restart keeps more Krylov vectors
    assert est(lib, [32] * 100, restart=120) > est(lib, [32] * 100, restart=60)
    # a boundary adds its nodes' arrays
    assert est(lib, [32] * 100, ns=4096) > e1


def test_estimate_rejects_invalid(lib):
    assert est(lib, [5]) == 0
    assert est(lib, [257]) == 0
    assert lib.fs_estimate_bytes(-1, None, 0, None) == 0
    assert lib.fs_estimate_bytes(0, None, 0, None) > 0   # an empty context still holds its status word
    assert est(lib, [32] * 4, prec=7) == 0                 # options fs_create would refuse
    assert est(lib, [32] * 4, restart=251) == 0


def test_server_argument_checks(lib):
    out = ctypes.c_void_p()
    assert lib.fs_server_create(ctypes.byref(out), 0, 1, 0) == _native.FS_EINVAL
    assert lib.fs_server_create(ctypes.byref(out), 1 << 30, 0, 0) == _native.FS_EINVAL
    assert lib.fs_server_create(None, 1 << 30, 1, 0) == _native.FS_EINVAL
    t = ctypes.c_uint64()
    rq = _native.fs_request()
    assert lib.fs_submit(None, ctypes.byref(rq), ctypes.byref(t)) == _native.FS_EINVAL
    assert lib.fs_poll(None, 1, None) == _native.FS_EINVAL
    assert lib.fs_server_wait(None, 1, None, 0.0) == _native.FS_EINVAL
    assert lib.fs_server_stats(None, None, None, None, None) == _native.FS_EINVAL
    lib.fs_server_destroy(None)


def test_server_create_without_a_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = ctypes.c_void_p()
    assert lib.fs_server_create(ctypes.byref(out), 1 << 30, 2, 0) == _native.FS_ECUDA
    assert not out.value
