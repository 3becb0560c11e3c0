"""The bounds-checked build (SB_CHECKED=1): it builds from the same sources,
exports the same entry points as the release build, reports which build it
is, and its status word decodes as include/sb.h states. No GPU needed: the
kernels' own tests of their indices run in tests/test_gpu_checked.py."""
import ctypes
import os
import re

import pytest

import paper_2402_14718_gb300 as sb
from paper_2402_14718_gb300 import _lib, build as _build
from tests.test_abi import declared_functions


@pytest.fixture(scope="module")
def libs():
    rel = ctypes.CDLL(_build.build())
    chk = ctypes.CDLL(_build.build(checked=True))
    for lib in (rel, chk):
        lib.sb_checked_build.restype = ctypes.c_int32
        lib.sb_check_bounds.restype = ctypes.c_int32
        lib.sb_check_bounds.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    return rel, chk


def test_checked_library_exports_every_declared_symbol(libs):
    for lib in libs:
        assert [n for n in declared_functions() if not hasattr(lib, n)] == []


def test_build_flag(libs):
    rel, chk = libs
    assert rel.sb_checked_build() == 0
    assert chk.sb_checked_build() == 1


def test_check_bounds_host_side(libs):
    """A NULL output is an argument error in both builds; the release build
    records nothing, so it answers without touching the device."""
    rel, chk = libs
    for lib in (rel, chk):
        assert lib.sb_check_bounds(None) == _lib.SB_ERR_ARG
    w = ctypes.c_uint64(123)
    assert rel.sb_check_bounds(ctypes.byref(w)) == _lib.SB_OK
    assert w.value == 0


def test_status_word_decoding():
    """module << 48 | site << 32 | index, the index as a signed 32-bit value."""
    assert sb.decode_bounds(0) is None
    assert sb.decode_bounds((1 << 48) | (1 << 32) | 1707) == ("step / energy kernels",
                                                               "CSR column", 1707)
    assert sb.decode_bounds((2 << 48) | (3 << 32) | 99) == ("factored kernels", "U row", 99)
    assert sb.decode_bounds((3 << 48) | (5 << 32) | 0xFFFFFFFF) == ("row-group kernel",
                                                                    "row-group union column", -1)
    assert sb.decode_bounds((2 << 48) | (2 << 32) | 5)[1] == "row-pointer pair"
    assert sb.decode_bounds((2 << 48) | (4 << 32) | 5)[1] == "group member"


def test_status_codes_match_the_header():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "sb.h")).read()
    assert int(re.search(r"SB_ERR_BOUNDS = (\d+)", text).group(1)) == _lib.SB_ERR_BOUNDS
    assert int(re.search(r"#define SB_OPT_TEST_BAD_COL (\d+)", text).group(1)) == \
        _lib.SB_OPT_TEST_BAD_COL
