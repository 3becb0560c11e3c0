"""The bounds-checked build on the GPU (child processes: one library each).

* Valid inputs: every step path (plain, one-replica, row-group, sign-byte,
  factored dSB / bSB) gives the release build's states and energies bit for
  bit, and no index is recorded.
* A planted column outside the state (SB_OPT_TEST_BAD_COL, a test hook of
  the checked build only): the untiled step kernel and the energy kernel
  record it (SB_ERR_BOUNDS, CSR column n + 7), read row 0 instead, and the
  device stays usable (a fresh context runs clean and matches the release
  build). Every read of the planted column in those two kernels goes through
  the check, so nothing is read outside the state."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(mode, out, checked):
    env = dict(os.environ)
    env["SB_LIBRARY"] = "checked" if checked else "release"
    r = subprocess.run([sys.executable, "-m", "tests.checked_child", mode, str(out)], cwd=ROOT,
                       env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-4000:]
    d = np.load(out)
    return d, json.loads(str(d["report"]))


def test_checked_build_matches_release_on_every_path(tmp_path):
    chk, rep_c = _child("paths", tmp_path / "c.npz", True)
    rel, rep_r = _child("paths", tmp_path / "r.npz", False)
    assert int(chk["checked"]) == 1 and int(rel["checked"]) == 0
    assert all(v is None for v in rep_c.values()), rep_c
    assert all(v is None for v in rep_r.values()), rep_r
    keys = [k for k in rel.files if k not in ("checked", "report")]
    assert len(keys) == 21
    for k in keys:
        assert np.array_equal(chk[k], rel[k]), k


def test_planted_column_is_recorded_and_skipped(tmp_path):
    d, rep = _child("bad", tmp_path / "b.npz", True)
    n = rep["n"]
    for when in ("after_step", "after_energy"):
        st, (module, site, idx), msg = rep[when]
        assert (module, site, idx) == ("step / energy kernels", "CSR column", n + 7), rep
        assert "outside" in msg
    assert rep["again"] is None     # the word was cleared by the first read
    assert rep["fresh"] is None
    rel, _ = _child("paths", tmp_path / "r.npz", False)
    assert np.array_equal(d["fresh_x"], rel["plain_bsb_r4_x"])
