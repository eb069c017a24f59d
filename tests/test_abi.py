"""The C-ABI library builds, loads and exports every entry point that include/sgks.h declares.
CPU only: no call reaches the GPU (argument validation fails before any CUDA call)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sgks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(sgks_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_2606_18073_gb300 as G
    G.build()
    return G._lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("sgks_create", "sgks_step", "sgks_solve", "sgks_destroy", "sgks_reset", "sgks_status",
              "sgks_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2606_18073_gb300 import _lib as L
    names = declared_functions()
    for f in names:
        assert hasattr(lib, f), f
    assert set(names) == set(L.exported_symbols())


def test_invalid_create_fails_before_touching_the_device(lib):
    from paper_2606_18073_gb300 import _lib as L
    h = C.c_void_p()
    op, reg, o = L.sgks_op(), L.sgks_reg(), L.sgks_options()
    rc = lib.sgks_create(C.byref(h), C.byref(op), C.byref(reg), None, 1.0, 10, 0, C.byref(o), None)
    assert rc == L.SGKS_ERR_INVALID and not h.value
    assert b"non-NULL" in lib.sgks_last_error(None)
    op.kind, op.m, op.n, op.val_dtype = L.SGKS_OP_CONV2D, 16, 16, L.SGKS_F32
    op.nx, op.ny, op.kh, op.kw, op.psf = 4, 4, 3, 3, C.c_void_p(16)
    reg.kind, reg.nx, reg.ny = L.SGKS_REG_GRAD2D, 4, 4
    rc = lib.sgks_create(C.byref(h), C.byref(op), C.byref(reg), C.c_void_p(16), -2.0, 10, 0, None, None)
    assert rc == L.SGKS_ERR_INVALID and b"lambda" in lib.sgks_last_error(None)
    rc = lib.sgks_create(C.byref(h), C.byref(op), C.byref(reg), C.c_void_p(16), 2.0, 5000, 0, None, None)
    assert rc == L.SGKS_ERR_INVALID and b"sketch_rows" in lib.sgks_last_error(None)
    lib.sgks_destroy(None)


def test_null_handles_are_rejected(lib):
    """Every call that takes a handle returns SGKS_ERR_INVALID for a NULL one, without a device call."""
    from paper_2606_18073_gb300 import _lib as L
    calls = {
        "sgks_reset": (None, None), "sgks_set_lambda": (None, 1.0), "sgks_backward": (None, None, None, None),
        "sgks_step": (None,), "sgks_solve": (None, 1, 0.0, None, None), "sgks_status": (None, None),
        "sgks_get_info": (None, None), "sgks_profile_steps": (None, 1, None, None, None),
        "sgks_profile_graph": (None, 1, None, None, None), "sgks_time_class": (None, 0, 1, None),
        "sgks_get_buffer": (None, 0, None, 0, None), "sgks_apply": (None, 0, None, None),
        "sgks_batch_reset": (None, None), "sgks_batch_step": (None,), "sgks_batch_solve": (None, 1, 0.0, None, None),
        "sgks_batch_get_x": (None, None), "sgks_batch_status": (None, None), "sgks_batch_layout": (None, None, None),
        "sgks_batch_profile_steps": (None, 1, None, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == L.SGKS_ERR_INVALID, name
    assert lib.sgks_batch_config(None, 0) == b""
    lib.sgks_batch_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2606_18073_gb300 import _lib as L
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        L._lib_saved = L._lib
        L._lib = None
        try:
            L.load(str(tmp_path / "missing.so"))
        finally:
            L._lib = L._lib_saved
