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


def test_body_arguments_are_validated_without_gpu(lib):
    """fs_create_with_body rejects an incomplete body, unknown end codes and
    attached ends without a body before any device call."""
    out = ctypes.c_void_p()
    ppf = (ctypes.c_int32 * 2)(16, 16)
    nodes = (ctypes.c_double * 12)(*([1.0, 0.0, 0.0] * 4))
    w = (ctypes.c_double * 4)(1.0, 1.0, 1.0, 1.0)
    D3 = ctypes.c_double * 3

    def body(n=4, radius=1.0, nod=nodes, force=(0.0, 0.0, 1.0)):
        return _native.fs_body(D3(0.0, 0.0, 0.0), radius, n, ctypes.cast(nod, ctypes.c_void_p) if nod else None,
                               ctypes.cast(nodes, ctypes.c_void_p), ctypes.cast(w, ctypes.c_void_p), D3(*force),
                               D3(0.0, 0.0, 0.0))

    def create(ends, b):
        e = (ctypes.c_int32 * 2)(*ends) if ends is not None else None
        return lib.fs_create_with_body(ctypes.byref(out), 2, ppf, e, 1.0, 1e-3, 1.0, 1e-3, None,
                                       ctypes.byref(b) if b is not None else None, None, None)

    assert create((1, 7), body()) == _native.FS_EINVAL                       # unknown end code
    assert b"end condition" in lib.fs_last_error()
    assert create((1, 0), None) == _native.FS_EINVAL                         # attached, no body
    assert b"no body" in lib.fs_last_error()
    assert create((0, 0), body(n=0)) == _native.FS_EINVAL                    # no surface nodes
    assert create((0, 0), body(radius=0.0)) == _native.FS_EINVAL             # no radius
    assert create((0, 0), body(nod=None)) == _native.FS_EINVAL               # missing nodes
    assert create((0, 0), body(force=(0.0, float("nan"), 0.0))) == _native.FS_EINVAL
    assert b"non-finite" in lib.fs_last_error()


def test_treecode_options_are_validated_without_gpu(lib):
    o = _native.fs_options()
    lib.fs_options_default(ctypes.byref(o))
    assert o.tree_order == 0 and o.tree_theta == 0.5
    out = ctypes.c_void_p()
    ppf = (ctypes.c_int32 * 1)(16)
    for order, theta in ((5, 0.5), (8, 1.0), (8, 0.0)):
        o.tree_order, o.tree_theta = order, theta
        assert lib.fs_create(ctypes.byref(out), 1, ppf, 1.0, 1e-3, 1.0, 1e-3, None, ctypes.byref(o),
                             None) == _native.FS_EINVAL
        assert b"tree" in lib.fs_last_error()


def test_step_options_are_validated_without_gpu(lib):
    """Every option outside its documented values is refused by fs_create
    before any CUDA call (an unknown precision would otherwise reach the
    flexible GMRES, whose outer Krylov space only FS_MIXED allocates)."""
    out = ctypes.c_void_p()
    ppf = (ctypes.c_int32 * 1)(16)
    bad = [("prec", 2), ("prec", -1), ("tol", 0.0), ("tol", 1.0), ("tol", float("nan")),
           ("inner_tol", 0.0), ("max_iter", 0), ("restart", 0), ("restart", 251),
           ("max_refine", 0), ("delta_over_L", -0.01), ("delta_over_L", float("inf")),
           ("lsb", 2), ("relax", -1), ("profile", 3), ("use_graph", 2),
           ("tile_override", 4), ("tile_override", -1), ("tc_lu", 2), ("autotune", 2)]
    for field, value in bad:
        o = _native.fs_options()
        lib.fs_options_default(ctypes.byref(o))
        setattr(o, field, value)
        assert lib.fs_create(ctypes.byref(out), 1, ppf, 1.0, 1e-3, 1.0, 1e-3, None, ctypes.byref(o),
                             None) == _native.FS_EINVAL, (field, value)
        assert not out.value
        msg = lib.fs_last_error()
        assert msg.startswith(b"fs_create:") and field.split("_")[0].encode() in msg, (field, msg)
    # the autotuner and graph cycles exclude each other
    o = _native.fs_options()
    lib.fs_options_default(ctypes.byref(o))
    o.autotune, o.use_graph = 1, 1
    assert lib.fs_create(ctypes.byref(out), 1, ppf, 1.0, 1e-3, 1.0, 1e-3, None, ctypes.byref(o),
                         None) == _native.FS_EINVAL
    assert b"autotune" in lib.fs_last_error()
    # the same checks guard the batch constructor
    o = _native.fs_options()
    lib.fs_options_default(ctypes.byref(o))
    o.prec = 5
    fps = (ctypes.c_int32 * 2)(1, 1)
    pp = (ctypes.c_int32 * 2)(16, 16)
    assert lib.fs_create_batch(ctypes.byref(out), 2, fps, pp, 1.0, 1e-3, 1.0, 1e-3, ctypes.byref(o),
                               None) == _native.FS_EINVAL
    assert lib.fs_last_error().startswith(b"fs_create_batch: prec")


def _header_structs():
    """name -> [(field, C type, array length)] for every typedef struct of
    the header, in declaration order."""
    text = open(os.path.join(ROOT, "include", "fibersolve.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*(?:fs_\w+\s*)?\{(.*?)\}\s*(fs_\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"((?:const )?[\w ]+?)\s*(\*?)\s*(\w+(?:\[\d+\])?(?:\s*,\s*\*?\s*\w+(?:\[\d+\])?)*)$", decl)
            assert m, decl
            ctype = m.group(1).strip() + (" *" if m.group(2) else "")
            for item in m.group(3).split(","):
                item = item.strip()
                ptr = item.startswith("*")
                item = item.lstrip("*").strip()
                n = 1
                am = re.match(r"(\w+)\[(\d+)\]", item)
                if am:
                    item, n = am.group(1), int(am.group(2))
                fields.append((item, ctype + (" *" if ptr else ""), n))
        out[name] = fields
    return out


def test_binding_struct_layouts_match_the_header():
    """Every struct the binding passes by reference has the header's fields,
    in order, with matching sizes (a silent layout mismatch would corrupt
    every call)."""
    sizes = {"double": 8, "int32_t": 4, "int64_t": 8, "size_t": 8}
    structs = _header_structs()
    checked = 0
    for name, fields in structs.items():
        cls = getattr(_native, name, None)
        if cls is None:
            continue
        py = cls._fields_
        assert [f[0] for f in py] == [f[0] for f in fields], name
        for (fname, ctype, n), (_, pytype) in zip(fields, py):
            if "*" in ctype:
                assert ctypes.sizeof(pytype) == ctypes.sizeof(ctypes.c_void_p), (name, fname)
            else:
                base = ctype.replace("const ", "").strip()
                assert ctypes.sizeof(pytype) == sizes[base] * n, (name, fname)
        checked += 1
    assert checked >= 7 and "fs_request" in structs


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every call raises ImportError: there is no
    CPU fallback behind the binding."""
    import paper_1602_05650_gb300 as fs
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "libfibersolve.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        fs.fs_options_default()
    with pytest.raises(ImportError):
        fs.fs_estimate_bytes([16, 16])


def test_header_is_plain_c_and_links(tmp_path):
    """A C99 program (no C++, no torch) includes the header, links the
    library and calls it: option defaults, a validation error with its
    message, the memory estimate."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    build.build()
    src = tmp_path / "client.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "fibersolve.h"
int main(void) {
    fs_options o;
    if (fs_options_default(&o) != FS_OK || o.prec != FS_MIXED) return 1;
    int32_t ppf[2] = {16, 5};
    fs_ctx *c = NULL;
    fs_status s = fs_create(&c, 2, ppf, 1.0, 1e-3, 1.0, 1e-3, NULL, &o, NULL);
    if (s != FS_EINVAL || c != NULL || strstr(fs_last_error(), "fiber 1") == NULL) return 2;
    if (strcmp(fs_status_str(s), "FS_EINVAL") != 0) return 3;
    if (fs_estimate_bytes(1, ppf, 0, &o) == 0 || fs_estimate_bytes(2, ppf, 0, &o) != 0) return 4;
    printf("ok\n");
    return 0;
}
''')
    lib_dir = os.path.dirname(_native.LIB_PATH)
    exe = tmp_path / "client"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                         "-I", os.path.join(ROOT, "include"), str(src), "-L", lib_dir, "-lfibersolve",
                         "-Wl,-rpath," + lib_dir, "-o", str(exe)], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and run.stdout.strip() == "ok", (run.returncode, run.stdout, run.stderr)
