"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point declared in include/*.h; the Python binding wraps each of them."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(bq_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1711_03836_gb300 import build

    return ctypes.CDLL(build.build())


def test_header_declares_entry_points():
    names = declared_functions()
    assert "bq_apply_dhop" in names and "bq_solve_cg" in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_1711_03836_gb300 import bqcd

    missing = [n for n in declared_functions() if n not in bqcd._SIGS]
    assert not missing, missing


def test_error_strings_without_gpu(lib):
    lib.bq_strerror.restype = ctypes.c_char_p
    assert lib.bq_strerror(0) == b"ok"
    assert b"argument" in lib.bq_strerror(1)
    # argument validation happens before any device call
    ctx = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(4, 4, 3, 4)
    assert lib.bq_create(ctypes.byref(ctx), dims, None) == 1
    assert not ctx.value
