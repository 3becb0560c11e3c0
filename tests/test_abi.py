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


def test_diagnostic_argument_errors():
    """sb_step_info and sb_gather_probe check their arguments before any device
    work."""
    import paper_2402_14718_gb300 as sb
    from paper_2402_14718_gb300 import _lib
    assert sb.lib.sb_step_info(None, None, None) == _lib.SB_ERR_ARG
    out = ctypes.c_double()
    for array_bytes, row_bytes, repeats, ptr in ((1 << 20, 100, 1, ctypes.byref(out)),
                                                 (1 << 20, 0, 1, ctypes.byref(out)),
                                                 (512, 512, 1, ctypes.byref(out)),
                                                 (1 << 20, 1024, 0, ctypes.byref(out)),
                                                 (1 << 20, 1024, 1, None)):
        assert sb.lib.sb_gather_probe(array_bytes, row_bytes, repeats, 1, ptr,
                                      None) == _lib.SB_ERR_ARG
    assert "sb_gather_probe" in sb.lib.sb_last_error().decode()


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


@pytest.mark.parametrize("case", ["diag", "range", "asym", "nan"])
def test_large_malformed_csr_reports_the_first_bad_row(case):
    """Rows are checked on several host threads when the CSR is large; the
    error still names the first bad row in row order (two faults planted in
    different parts of a 100,000-row chain)."""
    import paper_2402_14718_gb300 as sb
    from paper_2402_14718_gb300 import _lib
    n = 100000
    rows, cols = [], []
    for i in range(n):
        for j in (i - 1, i + 1):
            if 0 <= j < n:
                rows.append(i)
                cols.append(j)
    rowptr = np.zeros(n + 1, np.int32)
    np.add.at(rowptr, np.array(rows) + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    col = np.array(cols, np.int32)
    val = np.full(len(col), -1.0)
    lin = np.zeros(n)
    first, second = 70001, 90001
    if case == "diag":
        col[rowptr[first]] = first
        col[rowptr[second]] = second
        want, code = f"diagonal entry in row {first}", _lib.SB_ERR_CSR
    elif case == "range":
        col[rowptr[first + 1] - 1] = n + 5
        col[rowptr[second + 1] - 1] = n + 5
        want, code = f"column out of range in row {first}", _lib.SB_ERR_CSR
    elif case == "asym":
        val[rowptr[second]] = 0.5
        val[rowptr[first]] = 0.5
        want, code = f"not symmetric at ({first - 1}, {first})", _lib.SB_ERR_CSR
    else:
        lin[second] = np.nan
        val[rowptr[first]] = np.inf
        want, code = f"value not finite in row {first}", _lib.SB_ERR_ARG
    with pytest.raises(sb.SbError) as ei:
        sb.sb_create(n, rowptr, col, val, lin)
    assert ei.value.code == code
    assert want in sb.lib.sb_last_error().decode()


def test_binding_constants_match_the_header():
    """Every SB_OPT_* value and the status / variant / precision enums of
    include/sb.h equal the binding's constants."""
    from paper_2402_14718_gb300 import _lib
    text = open(os.path.join(ROOT, "include", "sb.h")).read()
    opts = dict(re.findall(r"^#define (SB_OPT_[A-Z0-9_]+) (\d+)", text, flags=re.M))
    assert opts, "no SB_OPT_* in the header"
    for name, value in opts.items():
        assert getattr(_lib, name) == int(value), name
    body = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for enum in re.findall(r"typedef enum\s*\{(.*?)\}", body, flags=re.S):
        value = -1
        for item in enum.split(","):
            item = item.strip()
            if not item:
                continue
            name, _, expr = item.partition("=")
            value = int(expr) if expr.strip() else value + 1
            assert getattr(_lib, name.strip()) == value, name
