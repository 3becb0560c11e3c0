"""The C-ABI library loads and exports every entry point include/sb.h declares;
host-side argument errors come back as status codes (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(sb_[a-z0-9_]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sb_create", "sb_run", "sb_energy", "sb_best", "sb_destroy",
                     "sb_last_error", "sb_create_batch", "sb_qubo_build", "sb_event_generate",
                     "sb_tracks"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2402_14718_gb300 as sb
    lib = ctypes.CDLL(sb.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_version_and_error_strings():
    import paper_2402_14718_gb300 as sb
    assert "sm_103a" in sb.sb_version()
    assert isinstance(sb.lib.sb_last_error(), bytes)


def test_host_argument_errors():
    import paper_2402_14718_gb300 as sb
    from paper_2402_14718_gb300 import _lib
    h = ctypes.c_void_p()
    # null output pointer
    assert sb.lib.sb_create(1, 0, None, None, None, None, 0, None) == _lib.SB_ERR_ARG
    # negative track count
    p = sb.event_params(n_tracks=-1)
    assert sb.lib.sb_event_generate(0, ctypes.byref(p), ctypes.byref(h)) == _lib.SB_ERR_ARG
    assert "range" in sb.lib.sb_last_error().decode()
    # bad precision code
    rp = np.array([0, 0], np.int32)
    lin = np.zeros(1)
    assert sb.lib.sb_create(1, 0, rp.ctypes.data, None, None, lin.ctypes.data, 7,
                            ctypes.byref(h)) == _lib.SB_ERR_ARG


@pytest.mark.parametrize("case", ["unsorted", "diag", "asym", "range", "rowptr"])
def test_malformed_csr_is_rejected_before_any_device_work(case):
    import paper_2402_14718_gb300 as sb
    from paper_2402_14718_gb300 import _lib
    rowptr = np.array([0, 2, 3, 4], np.int32)
    col = np.array([1, 2, 0, 0], np.int32)
    val = np.array([-1.0, 1.0, -1.0, 1.0])
    if case == "unsorted":
        col = np.array([2, 1, 0, 0], np.int32)
    elif case == "diag":
        col = np.array([0, 2, 0, 0], np.int32)
    elif case == "asym":
        val = np.array([-1.0, 1.0, -1.0, 0.5])
    elif case == "range":
        col = np.array([1, 3, 0, 0], np.int32)
    elif case == "rowptr":
        rowptr = np.array([0, 2, 3, 5], np.int32)
    with pytest.raises(sb.SbError) as ei:
        sb.sb_create(3, rowptr, col, val, np.zeros(3))
    assert ei.value.code == _lib.SB_ERR_CSR
