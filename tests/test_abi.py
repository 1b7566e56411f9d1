"""C-ABI checks that need no GPU: the library loads, exports every function that include/fe.h
declares, and rejects invalid arguments on the host before touching the device."""
import ctypes
import importlib.util
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fe.h")
LIB = os.path.join(ROOT, "paper_2607_02335_gb300", "libfe.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2607_02335_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fe_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fe_mesh_create", "fe_mesh_destroy", "fe_mesh_layout", "fe_gather", "fe_apply",
                     "fe_dss", "fe_diag", "fe_pairing", "fe_cg_solve", "fe_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_uses_the_same_names():
    from paper_2607_02335_gb300 import fe
    for name in declared_functions():
        assert hasattr(fe, name), name


def test_invalid_descriptors_rejected_on_host(lib):
    from paper_2607_02335_gb300 import fe
    for bad in (fe.fe_mesh_desc(2, 2, 2, 0, 0.0, 0, 0, 0), fe.fe_mesh_desc(2, 2, 2, 8, 0.0, 0, 0, 0),
                fe.fe_mesh_desc(0, 2, 2, 2, 0.0, 0, 0, 0), fe.fe_mesh_desc(2, 2, 2, 2, 0.1, 2, 0, 0),
                fe.fe_mesh_desc(2, 2, 2, 2, 0.5, 0, 0, 0), fe.fe_mesh_desc(2, 2, 2, 2, 0.0, 7, 0, 0)):
        h = ctypes.c_void_p()
        st = fe._lib.fe_mesh_create(ctypes.byref(bad), None, ctypes.byref(h))
        assert st == fe.FE_ERR_INVALID and h.value is None
        assert fe.fe_last_error()
    assert fe._lib.fe_mesh_create(None, None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_mesh_layout(None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_apply(None, 0, 0, None, None, 0, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_dss(None, 0, None, None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_diag(None, 0, None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_pairing(None, 0, None, None, None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_cg_solve(None, None, None, None, None, None) == fe.FE_ERR_INVALID
    assert fe._lib.fe_mesh_destroy(None) == fe.FE_OK
    # host-vector apply: every argument is checked before the device is touched
    y = (ctypes.c_void_p * 2)()
    ops = (ctypes.c_int * 2)(0, 1)
    assert fe._lib.fe_apply_host(None, 1, ops, None, y, 0, None) == fe.FE_ERR_INVALID
    assert fe.fe_last_error()
    for name, args in (("fe_mb_create", (None, None, None)), ("fe_amr_create", (None, None, None)),
                       ("fe_slab_face_pack", (None, 0, None, 0, None, None)),
                       ("fe_slab_face_add", (None, 0, None, 0, None, None)),
                       ("fe_slab_apply", (None, 0, 0, None, None, 0, None, None))):
        assert getattr(fe._lib, name)(*args) == fe.FE_ERR_INVALID, name


def test_binding_fails_loudly_without_library(tmp_path):
    src = os.path.join(ROOT, "paper_2607_02335_gb300", "fe.py")
    shutil.copy(src, tmp_path / "fe.py")
    spec = importlib.util.spec_from_file_location("fe_copy", tmp_path / "fe.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
