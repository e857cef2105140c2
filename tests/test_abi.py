"""The C ABI boundary, checked without a GPU: libwlr.so builds, loads, and exports
every function that include/*.h declares; the binding exposes the same names."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(wlr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1703_06303_gb300 import wlr
    return wlr


def test_header_declares_the_api():
    names = _declared()
    for n in ("wlr_create", "wlr_set_data", "wlr_set_init", "wlr_step", "wlr_solve",
              "wlr_objective", "wlr_get_result", "wlr_destroy", "wlr_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib.library_path())
    missing = [n for n in sorted(_declared()) if not hasattr(so, n)]
    assert not missing, missing


def test_binding_has_the_same_names(lib):
    for n in _declared():
        assert hasattr(lib, n), n
        assert n in lib.EXPORTED


def test_status_strings_and_host_validation(lib):
    # host-side argument checks run before any device call
    assert lib.wlr_status_string(0) == "WLR_OK"
    assert lib.wlr_status_string(4) == "WLR_ERR_NOT_SPD"
    with pytest.raises(lib.WlrError) as e:
        lib.wlr_create(10, 5, 6, 6)          # k > n
    assert e.value.status == lib.WLR_ERR_INVALID_ARG
    with pytest.raises(lib.WlrError) as e:
        lib.wlr_create(10, 8, 3, 2)          # r < k
    assert e.value.status == lib.WLR_ERR_INVALID_ARG
    with pytest.raises(lib.WlrError) as e:
        lib.wlr_create(1000, 200, 65, 70)    # k > 64
    assert e.value.status == lib.WLR_ERR_UNSUPPORTED
    with pytest.raises(lib.WlrError) as e:
        lib.wlr_create(1000, 200, 5, 40)     # r - k > 32
    assert e.value.status == lib.WLR_ERR_UNSUPPORTED


def test_batched_and_refine_host_validation(lib):
    import ctypes as ct
    # empty batch: nothing to do; negative counts and iteration numbers are refused before
    # any device call, as are a NULL handle array and NULL handles
    assert lib.wlr_solve_batched([], 5) == lib.WLR_OK
    failed = ct.c_int32(7)
    assert lib._lib.wlr_solve_batched(None, -1, 3, ct.byref(failed)) == lib.WLR_ERR_INVALID_ARG
    assert failed.value == -1
    assert lib._lib.wlr_solve_batched(None, 2, 3, ct.byref(failed)) == lib.WLR_ERR_INVALID_ARG
    arr = (ct.c_void_p * 2)(None, None)
    assert lib._lib.wlr_solve_batched(arr, 2, 3, None) == lib.WLR_ERR_INVALID_ARG
    assert lib._lib.wlr_solve_batched(arr, 0, -4, None) == lib.WLR_ERR_INVALID_ARG
    F0, F1 = ct.c_double(0), ct.c_double(0)
    assert lib._lib.wlr_refine(None, None, 0, 0, ct.byref(F0), ct.byref(F1)) == lib.WLR_ERR_INVALID_ARG


def test_no_oracle_import_in_product_code():
    # the product package never imports the oracle
    pkg = os.path.join(ROOT, "paper_1703_06303_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), path
