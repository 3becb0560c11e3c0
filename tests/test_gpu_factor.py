"""Factored coupling product (sb_set_factor): the conflict couplings of Eq. 13
as group sums over shared hits plus an exact residual.

Against the FP64 oracle (one step, 1e-5 as every FP32 step; the oracle runs
the plain CSR product), against the plain kernels (dSB: bit for bit, every
partial sum being a multiple of 1/4; rows left in plain form: bit for bit),
and on a generic random factor (any grouping is exact: the residual absorbs
the difference)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from oracle import ising, sb as osb
from tests import inputs
from tests.gpu_common import (compare_step, compare_step_elementwise, max_rel, oracle_c0,
                              workload_qubos)
from tests.test_gpu_parity import _oracle_J, _sched

pytestmark = pytest.mark.gpu
VNAME = {osb.ASB: "asb", osb.BSB: "bsb", osb.DSB: "dsb"}


def _fctx(q, prec, factor=True):
    ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, prec)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    if factor:
        member, couple, w, n_ids = sb.sb_qubo_factor(q)
        sb.sb_set_factor(ctx, n_ids, member, couple, w)
    return ctx


def _one_step(ctx, qo, prec, variant, R, seed, a_k, scale=0.8):
    c0 = oracle_c0(qo)
    x0, y0 = inputs.random_state(qo.n, R, seed, scale)
    sb.sb_set_state(ctx, x0, y0)
    sb.sb_advance(ctx, VNAME[variant], 1.0, c0, 0.5, 1, _sched([a_k]))
    xg, yg = sb.sb_get_state(ctx)
    J, h, _ = _oracle_J(qo, prec)
    a32 = float(np.float32(a_k))
    x64, y64 = x0.astype(np.float64), y0.astype(np.float64)
    xo, yo = osb.step(J, h, x64, y64, a32, 1.0, c0, 0.5, variant)
    xpre = osb.prewall_x(J, h, x64, y64, a32, 1.0, c0, 0.5, variant)
    compare_step_elementwise(J, h, x64, y64, a32, 1.0, c0, 0.5, variant, xg, yg, xo, yo, xpre)
    return compare_step(xg, yg, xo, yo, xpre)


@pytest.mark.parametrize("variant,R,rpw", [
    (osb.BSB, 4, -1), (osb.BSB, 64, -1), (osb.BSB, 256, -1), (osb.BSB, 256, 0), (osb.BSB, 512, -1),
    (osb.BSB, 128, -1), (osb.BSB, 128, 0), (osb.ASB, 32, -1), (osb.ASB, 256, -1), (osb.ASB, 256, 0),
    (osb.DSB, 16, -1), (osb.DSB, 64, -1), (osb.DSB, 256, -1), (osb.DSB, 1024, -1)])
@pytest.mark.parametrize("prec", [sb.SB_J_FP32, sb.SB_J_BF16])
def test_factor_one_step_against_oracle(variant, R, rpw, prec):
    """aSB / bSB with R a multiple of 128 run the row-group kernel over the
    extended CSR (U rows as columns); rows per warp 0 forces the dedicated
    factored kernel there; other R and dSB always take the dedicated one."""
    _, qc, _, qo = workload_qubos("event500")
    ctx = _fctx(qc, prec)
    sb.sb_set_option(ctx, sb.SB_OPT_ROWS_PER_WARP, rpw)
    info = sb.sb_factor_info(ctx)
    assert info["set"] == 1 and info["rows"] > 0.5 * qc.n
    _one_step(ctx, qo, prec, variant, R, 3 + R, 0.43)


@pytest.mark.parametrize("variant", ["bsb", "dsb"])
def test_factor_set_after_the_state_and_both_forms_agree(variant):
    """A factor set on a context that already holds a state (the x buffers grow
    to hold the U rows, keeping the state), then one step from the Philox start
    (no wall reached yet: a longer free run of this dense event hits walls
    within a few steps, where FP32 rounding may flip a wall decision): the
    row-group form and the dedicated factored kernel agree with each other to
    FP32 rounding (bSB) or bit for bit (dSB), and with the plain kernels."""
    _, qc, _, _ = workload_qubos("event1000")
    R = 256
    sched = _sched(np.float32(np.linspace(0, 1, 2000))[:1])
    outs = []
    for rpw, factor in ((-1, True), (0, True), (-1, False)):
        ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_BF16)
        sb.sb_set_option(ctx, sb.SB_OPT_ROWS_PER_WARP, rpw)
        sb.sb_run(ctx, variant, 1.0, 0.0, 0.5, 0, R, seed=15)
        if factor:
            member, couple, w, n_ids = sb.sb_qubo_factor(qc)
            sb.sb_set_factor(ctx, n_ids, member, couple, w)
        sb.sb_advance(ctx, variant, 1.0, 0.0, 0.5, 1, sched)
        outs.append(sb.sb_get_state(ctx))
    if variant == "dsb":
        for o in outs[1:]:
            assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1])
    else:
        # the field drives some rows onto the wall within one step; a wall
        # decision within rounding of |x| = 1 may differ, everything else agrees
        for o in outs[1:]:
            off = (np.abs(o[0]) < 1.0) & (np.abs(outs[0][0]) < 1.0)
            assert np.mean(~off & (np.abs(o[0]) != np.abs(outs[0][0]))) < 1e-4
            ref = outs[0][0].astype(np.float64)
            assert max_rel(np.where(off, o[0], 0), np.where(off, ref, 0)) < 1e-5
            ref = outs[0][1].astype(np.float64)
            assert max_rel(np.where(off, o[1], 0), np.where(off, ref, 0)) < 1e-5


@pytest.mark.parametrize("R", [16, 64, 256])
def test_factor_dsb_equals_plain_kernel_bit_for_bit(R):
    """dSB with couplings in multiples of 1/4: the factored sums are exact, so 25
    graph-replayed steps from the Philox start give the plain sign-byte kernel's
    state bit for bit."""
    _, qc, _, _ = workload_qubos("event1000")
    out = []
    for factor in (True, False):
        ctx = _fctx(qc, sb.SB_J_BF16, factor)
        sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 1)
        sb.sb_run(ctx, "dsb", 1.0, 0.0, 0.5, 25, R, seed=77)
        out.append(sb.sb_get_state(ctx))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("R", [64, 512])
def test_factor_dsb_whole_run_equals_plain_kernel_bit_for_bit(R):
    """Over a whole 1000-step dSB schedule (the bifurcation, then spins pinned on
    the walls, where the factored step writes back only what changed and x is
    updated in place), in one piece and enqueued as two halves, the factored
    states equal the plain sign-byte kernel's bit for bit; R = 512 runs two
    replica tiles."""
    _, qc, _, _ = workload_qubos("event1000")
    S = 1000
    a = np.linspace(0.0, 1.0, S)
    out = []
    for factor, halves in ((False, False), (True, False), (True, True)):
        ctx = _fctx(qc, sb.SB_J_BF16, factor)
        sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 1)
        sb.sb_run(ctx, "dsb", 1.0, 0.0, 0.5, 0, R, seed=31)
        if halves:
            sb.sb_advance(ctx, "dsb", 1.0, 0.0, 0.5, S // 2, _sched(a[:S // 2]))
            sb.sb_advance(ctx, "dsb", 1.0, 0.0, 0.5, S - S // 2, _sched(a[S // 2:]))
        else:
            sb.sb_advance(ctx, "dsb", 1.0, 0.0, 0.5, S, _sched(a))
        out.append(sb.sb_get_state(ctx))
    x, _ = out[0]
    assert np.mean(np.abs(x) == 1.0) > 0.5   # the run reaches the pinned phase
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])


def test_factor_dsb_large_blocks_fp32_u_rows_bit_for_bit():
    """Blocks of more than 256 members: BF16 cannot hold their U sums, so dSB
    takes FP32 U rows (still exact); 300 steps (into the phase where whole
    lanes sit on the wall) equal the plain sign-byte kernel's state bit for
    bit."""
    couple = np.array([[1, 1], [1, 0]], np.uint8)
    q, member = inputs.grouped_qubo(1200, 2, 4, couple, 1.0, 6, seed=12)
    out = []
    for factor in (True, False):
        ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_BF16)
        sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 1)
        if factor:
            sb.sb_set_factor(ctx, 4, member, couple, 1.0)
            info = sb.sb_factor_info(ctx)
            assert info["max_count"] > 256 and info["rows"] > q.n // 2
        sb.sb_run(ctx, "dsb", 1.0, 0.0, 0.5, 300, 64, seed=5)
        out.append(sb.sb_get_state(ctx))
    assert np.mean(np.abs(out[0][0]) == 1.0) > 0.5
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_factor_rows_left_plain_equal_plain_kernel():
    """Couplings that BF16 cannot hold exactly leave every residual inexact: all
    rows stay in plain form, and the factored kernel then runs the CSR-order FMA
    chain of the plain kernels (same states bit for bit)."""
    q = inputs.random_qubo(700, 12, seed=8, values=(-0.731, 0.377, 1.234))
    rng = np.random.default_rng(4)
    member = rng.integers(0, 90, size=(q.n, 2)).astype(np.int32)
    couple = np.array([[1, 1], [1, 0]], np.uint8)
    x0, y0 = inputs.random_state(q.n, 128, 5, 0.7)
    outs = []
    for factor in (True, False):
        ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_BF16)
        sb.sb_set_option(ctx, sb.SB_OPT_ROWS_PER_WARP, 0)
        if factor:
            sb.sb_set_factor(ctx, 90, member, couple, 1.0)
            assert sb.sb_factor_info(ctx)["rows"] == 0
        sb.sb_set_state(ctx, x0, y0)
        sb.sb_advance(ctx, "bsb", 1.0, 0.3, 0.5, 6, _sched(np.linspace(0, 1, 6)))
        outs.append(sb.sb_get_state(ctx))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("variant", [osb.BSB, osb.DSB])
def test_generic_random_factor_against_oracle(variant):
    """A factor with no relation to the couplings (random blocks, K = 3, a random
    symmetric pattern): the residual takes up the whole difference and the step
    still matches the oracle's plain CSR product."""
    q = inputs.random_qubo(900, 20, seed=11, values=(-1.0, 0.5, 2.0), lin_low=-1, lin_high=1)
    rng = np.random.default_rng(12)
    member = rng.integers(-1, 40, size=(q.n, 3)).astype(np.int32)
    couple = np.array([[1, 0, 1], [0, 1, 1], [1, 1, 0]], np.uint8)
    ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_FP32)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    sb.sb_set_factor(ctx, 40, member, couple, 0.5)
    info = sb.sb_factor_info(ctx)
    assert info["set"] == 1
    R = 64
    _one_step(ctx, q, sb.SB_J_FP32, variant, R, 21, 0.6)
    # removing the factor returns to the plain kernels
    sb.sb_set_factor(ctx, 0, None, None, 0.0)
    assert sb.sb_factor_info(ctx)["set"] == 0
    _one_step(ctx, q, sb.SB_J_FP32, variant, R, 22, 0.6)


def test_factor_batch_matches_single_events():
    """Three events in one context, hit ids offset per event: each event's slice
    of a 15-step factored bSB run equals that event's own factored run."""
    names = ["event100", "event500"]
    qs = [workload_qubos(nm)[1] for nm in names] + [workload_qubos("event100")[1]]
    facs = [sb.sb_qubo_factor(q) for q in qs]
    off, members = 0, []
    for (m, _, _, n_ids) in facs:
        members.append(np.where(m >= 0, m + off, -1))
        off += n_ids
    R, S = 64, 15
    states = [inputs.random_state(q.n, R, 40 + k, 0.5) for k, q in enumerate(qs)]
    ctxb = sb.sb_create_batch([(q.rowptr, q.col, q.val, q.lin) for q in qs], sb.SB_J_BF16)
    sb.sb_set_factor(ctxb, off, np.concatenate(members), facs[0][1], facs[0][2])
    sb.sb_set_state(ctxb, np.concatenate([s[0] for s in states]), np.concatenate([s[1] for s in states]))
    sched = _sched(np.float32(np.linspace(0, 1, S)))
    sb.sb_advance(ctxb, "bsb", 1.0, 0.0, 0.5, S, sched)
    xb, yb = sb.sb_get_state(ctxb)
    row0 = 0
    for q, (x0, y0) in zip(qs, states):
        ctx = _fctx(q, sb.SB_J_BF16)
        sb.sb_set_state(ctx, x0, y0)
        sb.sb_advance(ctx, "bsb", 1.0, 0.0, 0.5, S, sched)
        x, y = sb.sb_get_state(ctx)
        assert np.array_equal(xb[row0:row0 + q.n], x) and np.array_equal(yb[row0:row0 + q.n], y)
        row0 += q.n


def test_factor_argument_errors():
    _, qc, _, _ = workload_qubos("event100")
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin)
    member, couple, w, n_ids = sb.sb_qubo_factor(qc)
    assert couple.tolist() == [[1, 1, 0], [1, 1, 1], [0, 1, 1]] and w == 1.0
    for args in ((n_ids, member, np.array([[1, 1, 0], [0, 1, 1], [0, 1, 1]], np.uint8), w),  # asymmetric
                 (n_ids, member, couple, 0.3),                        # -w/4 not exact in FP32
                 (int(member.max()), member, couple, w),              # ids beyond n_ids
                 (n_ids, member, couple * 2, w)):                     # not 0/1
        with pytest.raises(sb.SbError) as ei:
            sb.sb_set_factor(ctx, *args)
        assert ei.value.code == 1
    assert sb.sb_factor_info(ctx)["set"] == 0
    # hit ids shared by two events of a batch
    ctxb = sb.sb_create_batch([(qc.rowptr, qc.col, qc.val, qc.lin)] * 2)
    with pytest.raises(sb.SbError) as ei:
        sb.sb_set_factor(ctxb, n_ids, np.concatenate([member, member]), couple, w)
    assert ei.value.code == 1 and "more than one event" in str(ei.value)


def test_factor_short_horizon_free_running():
    """20 graph-replayed bSB steps from the Philox start on the linear ramp,
    factored product against the free-running oracle (1e-4, as for the plain
    kernels' 20-step horizon)."""
    _, qc, _, qo = workload_qubos("event500")
    R, S = 32, 20
    ctx = _fctx(qc, sb.SB_J_FP32)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 1)
    c0 = oracle_c0(qo)
    sched = np.float32(np.linspace(0.0, 1.0, 1000))[:S]
    sb.sb_run(ctx, "bsb", 1.0, c0, 0.5, 0, R, seed=9)
    sb.sb_advance(ctx, "bsb", 1.0, c0, 0.5, S, _sched(sched))
    xg, yg = sb.sb_get_state(ctx)
    J, h, _ = ising.to_ising(qo)
    xo, yo = osb.init_state(9, qo.n, R)
    res = osb.run(J, h, xo, yo, sched.astype(np.float64), 1.0, c0, 0.5, osb.BSB)
    assert max_rel(xg, res.x) < 1e-4 and max_rel(yg, res.y) < 1e-4


def test_factor_full_size_event1000_sampled():
    """The bench workload (1000 tracks, R = 256, BF16 J): one factored step from a
    random full-size state, 300 sampled rows against the oracle, for bSB and dSB."""
    _, qc, _, qo = workload_qubos("event1000")
    R = 256
    ctx = _fctx(qc, sb.SB_J_BF16)
    info = sb.sb_factor_info(ctx)
    assert info["rows"] > 0.85 * qc.n and info["max_count"] <= 256
    c0 = oracle_c0(qo)
    x0, y0 = inputs.random_state(qo.n, R, 78, 0.9)
    J, h, _ = _oracle_J(qo, sb.SB_J_BF16)
    rows = np.random.default_rng(3).choice(qo.n, 300, replace=False)
    x64, y64 = x0.astype(np.float64), y0.astype(np.float64)
    for variant in (osb.BSB, osb.DSB):
        sb.sb_set_state(ctx, x0, y0)
        sb.sb_advance(ctx, VNAME[variant], 1.0, c0, 0.5, 1, _sched([0.6]))
        xg, yg = sb.sb_get_state(ctx)
        a32 = float(np.float32(0.6))
        xo, yo = osb.step_rows(J, h, x64, y64, rows, a32, 1.0, c0, 0.5, variant)
        xpre = osb.prewall_x(J, h, x64, y64, a32, 1.0, c0, 0.5, variant, rows=rows)
        compare_step(xg[rows], yg[rows], xo, yo, xpre)
        compare_step_elementwise(J, h, x64, y64, a32, 1.0, c0, 0.5, variant, xg[rows], yg[rows],
                                 xo, yo, xpre, rows=rows)
