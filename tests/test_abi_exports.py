"""The C-ABI library builds for sm_103a and exports every entry point include/duwp.h declares
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "duwp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(duwp_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2305_12071_gb300 import build as B
    return B.build()


def test_header_and_binding_agree():
    from paper_2305_12071_gb300 import duwp
    assert _declared() == sorted(duwp.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_error_strings_without_device(libpath):
    lib = ctypes.CDLL(libpath)
    lib.duwp_error_string.restype = ctypes.c_char_p
    assert lib.duwp_error_string(0) == b"ok"
    assert b"overflow" in lib.duwp_error_string(-7)


def test_struct_layout_matches_header():
    # the ctypes mirror of duwp_params has the C layout: 8-byte alignment, no hidden padding
    from paper_2305_12071_gb300 import duwp
    assert ctypes.sizeof(duwp.Params) % 8 == 0
    assert duwp.Params.seed.offset % 8 == 0
    assert ctypes.sizeof(duwp.State) == 40


def test_binding_refuses_without_library(tmp_path):
    from paper_2305_12071_gb300 import duwp
    with pytest.raises(RuntimeError):
        duwp._lib_backup = duwp._lib
        duwp._lib = None
        try:
            duwp.load(str(tmp_path / "missing.so"))
        finally:
            duwp._lib = duwp._lib_backup
