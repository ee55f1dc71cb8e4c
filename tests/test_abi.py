"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function declared in include/pfmbem.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1910_10863_gb300 import build, pfmbem
    if not os.path.exists(pfmbem.LIB_PATH):
        build.build()
    return pfmbem.LIB_PATH


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pfmbem.h")).read()
    return sorted(set(re.findall(r"\b(pfmbem_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_api():
    names = declared_symbols()
    for must in ("pfmbem_create", "pfmbem_matvec", "pfmbem_solve", "pfmbem_field", "pfmbem_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_rejects_bad_arguments_without_gpu(libpath):
    from paper_1910_10863_gb300 import pfmbem
    L = pfmbem.lib()
    h = ctypes.c_void_p()
    # null output handle / nonsense sizes are rejected before any device work
    assert L.pfmbem_create(0, None, None, 1.0, 0, 1.0, 1.0, 1.0, 0.0, None, None, ctypes.byref(h)) == 1
    assert L.pfmbem_create(1, None, None, -1.0, 0, 1.0, 1.0, 1.0, 0.0, None, None, None) == 1
    assert L.pfmbem_matvec(None, None, None, 0) == 1
