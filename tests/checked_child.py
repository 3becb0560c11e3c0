"""Child process of tests/test_gpu_checked.py (not a test module): runs the
step kernels on one small event with the library that SB_LIBRARY selects
(the release build, or SB_LIBRARY=checked for the bounds-checked build) and
stores states, energies and what sb_check_bounds reported in an .npz file.
One library per process: the binding loads one.

  python -m tests.checked_child paths OUT.npz   every step path, valid inputs
  python -m tests.checked_child bad OUT.npz     one planted column (checked build only)
"""
import json
import sys

import numpy as np

import paper_2402_14718_gb300 as sb
from paper_2402_14718_gb300.workloads import WORKLOADS

# (name, variant, replicas, factored, precision): the plain untiled kernel,
# the one-replica kernel, the row-group kernel, the sign-byte kernel and the
# factored kernels (dedicated dSB / bSB, and bSB through the extended CSR)
PATHS = [("plain_bsb_r4", "bsb", 4, False, sb.SB_J_FP32),
         ("r1_bsb", "bsb", 1, False, sb.SB_J_FP32),
         ("rw_bsb_r128", "bsb", 128, False, sb.SB_J_BF16),
         ("dsb16_r64", "dsb", 64, False, sb.SB_J_BF16),
         ("fac_dsb_r64", "dsb", 64, True, sb.SB_J_BF16),
         ("fac_bsb_r64", "bsb", 64, True, sb.SB_J_BF16),
         ("fac_bsb_r128", "bsb", 128, True, sb.SB_J_BF16)]


def event_qubo():
    w = WORKLOADS["event100"]
    ev = sb.sb_event_generate(w["seed"], sb.event_params(n_tracks=w["n_tracks"],
                                                         noise_frac=w["noise_frac"]))
    return sb.sb_qubo_build(ev, sb.build_params(**w["cuts"]))


def run_paths(q):
    out, report = {}, {}
    for name, variant, R, factored, prec in PATHS:
        ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, prec)
        if factored:
            member, couple, wgt, n_ids = sb.sb_qubo_factor(q)
            sb.sb_set_factor(ctx, n_ids, member, couple, wgt)
        sb.sb_run(ctx, variant, 1.0, 0.0, 0.5, 60, R, seed=9)
        x, y = sb.sb_get_state(ctx)
        T, E, r = sb.sb_best(ctx)
        out[name + "_x"], out[name + "_y"] = x, y
        out[name + "_E"] = np.asarray(E, np.float64)
        report[name] = sb.sb_check_bounds()
        sb.sb_destroy(ctx)
    return out, report


def run_bad(q):
    """Column p of row `row` is overwritten with n + 7 on the device; one plain
    bSB step (R = 4: the untiled kernel) and the energy readout must record it
    and read row 0 instead."""
    row = int(np.argmax(np.diff(q.rowptr) > 0))
    p = int(q.rowptr[row])
    ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_FP32)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    sb.sb_set_option(ctx, sb.SB_OPT_TEST_BAD_COL, p)
    report = {"n": q.n}
    sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 1, 4, seed=9)
    report["after_step"] = sb.sb_check_bounds()
    report["again"] = sb.sb_check_bounds()
    sb.sb_energy(ctx)
    report["after_energy"] = sb.sb_check_bounds()
    sb.sb_destroy(ctx)
    # a fresh context on the same device runs clean afterwards
    ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_FP32)
    sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 60, 4, seed=9)
    x, _ = sb.sb_get_state(ctx)
    report["fresh"] = sb.sb_check_bounds()
    sb.sb_destroy(ctx)
    return {"fresh_x": x}, report


def main(mode, path):
    q = event_qubo()
    out, report = run_paths(q) if mode == "paths" else run_bad(q)
    out["checked"] = np.array(int(sb.sb_checked_build()))
    out["report"] = np.array(json.dumps(report))
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
