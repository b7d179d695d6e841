"""C ABI checks that need no GPU: the library builds and loads, exports every
entry point the headers declare, and rejects bad arguments before touching
the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in ("st.h", "st_stages.h"):
        with open(os.path.join(ROOT, "include", h)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:st_status|const\s+char\s*\*|size_t)\s*(st_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_headers_declare_entry_points():
    names = _declared()
    for n in ("st_plan_create", "st_inv_trans", "st_dir_trans", "st_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(st_mod):
    lib = st_mod.load()
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(st_mod):
    assert _declared() <= set(st_mod.SIGNATURES), _declared() - set(st_mod.SIGNATURES)


def test_argument_errors_without_device(st_mod):
    lib = st_mod.load()
    ST_ERR_ARG = 1
    assert lib.st_plan_create(None, 31, None, 0, 1, None) == ST_ERR_ARG
    h = ctypes.c_void_p()
    bad = st_mod._GridDesc(0, 31, 64)                      # odd nlat
    assert lib.st_plan_create(ctypes.byref(h), 31, ctypes.byref(bad), 0, 1, None) == ST_ERR_ARG
    assert h.value is None
    good = st_mod._GridDesc(0, 32, 64)
    assert lib.st_plan_create(ctypes.byref(h), 0, ctypes.byref(good), 0, 1, None) == ST_ERR_ARG
    assert lib.st_plan_create(ctypes.byref(h), 31, ctypes.byref(good), 9, 1, None) == ST_ERR_ARG
    assert lib.st_plan_create(ctypes.byref(h), 31, ctypes.byref(good), 0, 0, None) == ST_ERR_ARG
    assert lib.st_inv_trans(None, None, None, 1, None) == ST_ERR_ARG
    assert lib.st_dir_trans(None, None, None, 1, None) == ST_ERR_ARG
    assert lib.st_plan_query(None, None) == ST_ERR_ARG
    assert lib.st_plan_destroy(None) == 0
    assert lib.st_gauss_nodes(1, None, None, None) == ST_ERR_ARG
    assert lib.st_legendre_values(-1, None, 1, None, None) == ST_ERR_ARG
    assert lib.st_status_string(4) == b"device-side wait timed out"
    assert lib.st_plan_inject(None, 1, 100) == ST_ERR_ARG
    assert lib.st_plan_create_shared(None, None, 1, None) == ST_ERR_ARG
    assert lib.st_batch_create(None, None, 0) == ST_ERR_ARG
    assert lib.st_inv_trans_static(None, None, None, 1, None) == ST_ERR_ARG


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1908_06096_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    text = fh.read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "sht_oracle" not in text and "liboracle" not in text, f
