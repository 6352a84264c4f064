"""The C-ABI library builds, loads and exports every symbol that
include/fibersolve.h declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_1602_05650_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fibersolve.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:fs_status|void|uint64_t|size_t|const char \*)\s*\*?\s*(fs_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for must in ["fs_create", "fs_stokeslet_apply", "fs_build_precond", "fs_step", "fs_set_state",
                 "fs_get_state", "fs_destroy", "fs_last_error"]:
        assert must in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    # and the binding declares a signature for each of them
    assert set(declared_symbols()) <= set(_native.exported_symbols())


def test_options_default_and_errors_without_gpu(lib):
    o = _native.fs_options()
    assert lib.fs_options_default(ctypes.byref(o)) == 0
    assert o.prec == _native.FS_MIXED and o.tol == 1e-8 and o.restart == 60
    assert o.inner_tol == 1e-6 and o.relax == 1
    assert lib.fs_options_default(None) == _native.FS_EINVAL
    assert b"NULL" in lib.fs_last_error()
    # argument validation happens before any device call
    out = ctypes.c_void_p()
    assert lib.fs_create(ctypes.byref(out), -1, None, 1.0, 1e-3, 1.0, 1e-3, None, None, None) == _native.FS_EINVAL
    bad = (ctypes.c_int32 * 1)(3)
    assert lib.fs_create(ctypes.byref(out), 1, bad, 1.0, 1e-3, 1.0, 1e-3, None, None, None) == _native.FS_EINVAL
    assert lib.fs_status_str(4) == b"FS_ENOTCONV"
