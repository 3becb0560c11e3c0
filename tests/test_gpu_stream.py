"""Streamed step kernel (SB_OPT_STREAM): bulk-copied neighbour rows in a
shared-memory ring, consumer warps accumulating in CSR order.

It runs the same FMA sequence per (row, replica) as the untiled kernel, so the
two must agree bit for bit; one step is also checked against the FP64 oracle
(1e-5, as for every FP32 step)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from oracle import sb as osb
from tests import inputs
from tests.gpu_common import compare_step, workload_qubos, oracle_c0
from tests.test_gpu_parity import _oracle_J, _sched

pytestmark = pytest.mark.gpu
VARIANTS = ["asb", "bsb", "dsb"]


def _run(q, prec, variant, R, steps, stream, seed=3, graph=1, state=None):
    ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, prec)
    sb.sb_set_option(ctx, sb.SB_OPT_STREAM, stream)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, graph)
    dt = 0.1 if variant == "asb" else 0.5
    if state is None:
        sb.sb_run(ctx, variant, 1.0, 0.0, dt, steps, R, seed=seed)
    else:
        sb.sb_set_state(ctx, *state)
        sched = _sched(np.float32(np.linspace(0, 1, steps)))
        sb.sb_advance(ctx, variant, 1.0, 0.0, dt, steps, sched)
    x, y = sb.sb_get_state(ctx)
    return ctx, x, y


def _same(q, prec, variant, R, steps, **kw):
    _, xs, ys = _run(q, prec, variant, R, steps, 1, **kw)
    _, xu, yu = _run(q, prec, variant, R, steps, 0, **kw)
    assert np.array_equal(xs, xu) and np.array_equal(ys, yu)
    return xs


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", [sb.SB_J_FP32, sb.SB_J_BF16])
@pytest.mark.parametrize("R", [64, 128, 256, 512, 96])
def test_stream_and_untiled_bit_identical(variant, prec, R):
    """R = 64 / 128 / 256 use replica tiles of that width, 512 two tiles of 256,
    96 is not a multiple of 64 and falls back to the untiled kernel."""
    _, qc, _, _ = workload_qubos("event500")
    _same(qc, prec, variant, R, 25)


@pytest.mark.parametrize("variant", VARIANTS)
def test_stream_one_step_against_oracle(variant):
    _, qc, _, qo = workload_qubos("event100")
    R = 64
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_FP32)
    sb.sb_set_option(ctx, sb.SB_OPT_STREAM, 1)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    c0 = oracle_c0(qo)
    x0, y0 = inputs.random_state(qo.n, R, 11 + len(variant), 0.8)
    sb.sb_set_state(ctx, x0, y0)
    a_k = 0.37
    sb.sb_advance(ctx, variant, 1.0, c0, 0.5, 1, _sched([a_k]))
    xg, yg = sb.sb_get_state(ctx)
    J, h, _ = _oracle_J(qo, sb.SB_J_FP32)
    v = {"asb": osb.ASB, "bsb": osb.BSB, "dsb": osb.DSB}[variant]
    a32 = float(np.float32(a_k))
    x64, y64 = x0.astype(np.float64), y0.astype(np.float64)
    xo, yo = osb.step(J, h, x64, y64, a32, 1.0, c0, 0.5, v)
    xpre = osb.prewall_x(J, h, x64, y64, a32, 1.0, c0, 0.5, v)
    compare_step(xg, yg, xo, yo, xpre)


def test_stream_ragged_sizes_and_empty_rows():
    """N not a multiple of the 32-row block, isolated rows (empty CSR rows,
    whose blocks may hold no column at all), and a direct (non-graph) run."""
    q = inputs.random_qubo(1000, 7, seed=21)
    rp = np.concatenate([q.rowptr, np.full(45, q.rowptr[-1])]).astype(np.int32)
    lin = np.concatenate([q.lin, np.linspace(-0.4, 0.4, 45)])
    qe = inputs.QuboArrays(1045, rp, q.col, q.val, lin)
    for variant in VARIANTS:
        _same(qe, sb.SB_J_FP32, variant, 64, 17, graph=0)
        _same(qe, sb.SB_J_BF16, variant, 128, 9)
    # every row isolated: one all-padding stage per block
    qz = inputs.QuboArrays(70, np.zeros(71, np.int32), np.zeros(0, np.int32),
                           np.zeros(0), np.linspace(-1, 1, 70))
    _same(qz, sb.SB_J_FP32, "bsb", 64, 12)


def test_stream_dense_rows_and_fallback():
    """Rows of high degree give large per-block J spans (fewer ring stages);
    a complete graph's J span does not fit shared memory and the untiled kernel
    runs instead. Both agree with the untiled kernel bit for bit."""
    qd = inputs.random_qubo(600, 300, seed=5, values=(-1.0, 0.5, 2.0))
    _same(qd, sb.SB_J_FP32, "bsb", 256, 10)
    _same(qd, sb.SB_J_BF16, "dsb", 64, 10)
    qk = inputs.random_qubo(1300, 1299, seed=6)
    _same(qk, sb.SB_J_FP32, "bsb", 64, 4)


def test_stream_batch_matches_single_events():
    """Row blocks of a batched context may span two events; per-event c0 and
    rows still follow each event's own trajectory."""
    qs = [workload_qubos("event100")[1], inputs.random_qubo(300, 9, seed=3),
          inputs.random_qubo(77, 4, seed=4)]
    R, S = 128, 20
    states = [inputs.random_state(q.n, R, 50 + k, 0.5) for k, q in enumerate(qs)]
    ctxb = sb.sb_create_batch([(q.rowptr, q.col, q.val, q.lin) for q in qs])
    sb.sb_set_option(ctxb, sb.SB_OPT_STREAM, 1)
    sb.sb_set_state(ctxb, np.concatenate([s[0] for s in states]),
                    np.concatenate([s[1] for s in states]))
    sched = _sched(np.float32(np.linspace(0, 1, S)))
    sb.sb_advance(ctxb, "bsb", 1.0, 0.0, 0.5, S, sched)
    xb, yb = sb.sb_get_state(ctxb)
    row0 = 0
    for q, (x0, y0) in zip(qs, states):
        ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin)
        sb.sb_set_state(ctx, x0, y0)
        sb.sb_advance(ctx, "bsb", 1.0, 0.0, 0.5, S, sched)
        x, y = sb.sb_get_state(ctx)
        assert np.array_equal(xb[row0:row0 + q.n], x) and np.array_equal(yb[row0:row0 + q.n], y)
        row0 += q.n


def test_stream_full_size_event1000():
    """The 1000-track workload at R = 256 with BF16 J (the bench launch shape):
    streamed and untiled states agree bit for bit after 6 graph-replayed steps,
    and the readout reports no pipeline time-out."""
    _, qc, _, _ = workload_qubos("event1000")
    ctx, xs, ys = _run(qc, sb.SB_J_BF16, "bsb", 256, 8, 1)
    _, xu, yu = _run(qc, sb.SB_J_BF16, "bsb", 256, 8, 0)
    assert np.array_equal(xs, xu) and np.array_equal(ys, yu)
    T, E, r = sb.sb_best(ctx)
    assert 0 <= r < 256 and np.isfinite(E)


def test_stream_wait_runs_out_and_the_context_recovers():
    """The bounded-wait path of the streamed kernel. With the test hook, CTA 0's
    producer leaves its first ring stage unissued (no arrival, no copy), so the
    consumers' wait for it runs out after 1 ms; the kernel returns, the next
    synchronising call reports SB_ERR_TIMEOUT once, and a normal run on the
    same context then matches the untiled kernel bit for bit and the oracle."""
    _, qc, _, qo = workload_qubos("event100")
    R = 64
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_FP32)
    sb.sb_set_option(ctx, sb.SB_OPT_STREAM, 1)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    sb.sb_set_option(ctx, sb.SB_OPT_WAIT_NS, 1_000_000)
    sb.sb_set_option(ctx, sb.SB_OPT_TEST_SKIP_STAGE, 0)
    sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 2, R, seed=5)
    with pytest.raises(sb.SbError) as ei:
        sb.sb_get_state(ctx)
    assert ei.value.code == 5 and "gave up waiting" in str(ei.value)   # SB_ERR_TIMEOUT
    # reported once: the flag is cleared
    sb.sb_set_option(ctx, sb.SB_OPT_TEST_SKIP_STAGE, -1)
    sb.sb_set_option(ctx, sb.SB_OPT_WAIT_NS, 2_000_000_000)
    c0 = oracle_c0(qo)
    x0, y0 = inputs.random_state(qo.n, R, 29, 0.8)
    sb.sb_set_state(ctx, x0, y0)
    sb.sb_advance(ctx, "bsb", 1.0, c0, 0.5, 1, _sched([0.45]))
    xg, yg = sb.sb_get_state(ctx)
    ref = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_FP32)
    sb.sb_set_option(ref, sb.SB_OPT_GRAPH, 0)
    sb.sb_set_state(ref, x0, y0)
    sb.sb_advance(ref, "bsb", 1.0, c0, 0.5, 1, _sched([0.45]))
    xu, yu = sb.sb_get_state(ref)
    assert np.array_equal(xg, xu) and np.array_equal(yg, yu)
    J, h, _ = _oracle_J(qo, sb.SB_J_FP32)
    a32 = float(np.float32(0.45))
    x64, y64 = x0.astype(np.float64), y0.astype(np.float64)
    xo, yo = osb.step(J, h, x64, y64, a32, 1.0, c0, 0.5, osb.BSB)
    compare_step(xg, yg, xo, yo, osb.prewall_x(J, h, x64, y64, a32, 1.0, c0, 0.5, osb.BSB))
