"""The C-ABI library builds for sm_103a, loads and exports every function declared in include/imexds.h.
No device calls (runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "imexds.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(imexds_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_00705_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "imexds_create" in names and "imexds_run_to" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_2211_00705_gb300 import imexds
    assert sorted(imexds.EXPORTED) == declared_functions()


def test_status_strings_without_device(lib):
    lib.imexds_status_string.restype = ctypes.c_char_p
    assert lib.imexds_status_string(0) == b"ok"
    assert b"capacity" in lib.imexds_status_string(9)
