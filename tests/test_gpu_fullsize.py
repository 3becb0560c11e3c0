"""Parity at the full sizes of the 10k-track and 512-event workloads, in the
step-kernel configurations the bench times there, on sampled outputs.

* 10k-track event (N = 472,812, R = 128, BF16 J): the host builder's CSR equals
  the oracle builder's bit for bit at this size; one step from a random
  full-size state, 300 sampled rows against the FP64 oracle (1e-5), for bSB
  (row groups) and dSB (sign bytes), default and 32 rows per CTA.
* 512 uneven events in one context (R = 64, BF16 J, dSB): three sampled
  events, built again by the oracle builder (bit-exact CSR); the batch's Philox
  start equals the oracle's start of each event alone, bit for bit; one step of
  the whole batch from a random full-size state against the oracle step of
  each sampled event (1e-5). The step starts from identical values on both
  sides, so sgn(x) agrees exactly (a free-running dSB comparison at this size
  would meet positions within rounding of zero)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from paper_2402_14718_gb300.workloads import BATCH512, batch512_tracks
from oracle import events as oev, ising, qubo as oq, sb as osb
from tests import inputs
from tests.gpu_common import compare_step, oracle_params, workload_qubos, oracle_c0
from tests.test_gpu_parity import _oracle_J, _sched

pytestmark = pytest.mark.gpu


def test_full_size_event10k_builder_and_step_sampled():
    _, qc, _, qo = workload_qubos("event10k")
    assert qc.n == qo.n
    assert np.array_equal(qc.rowptr, qo.rowptr) and np.array_equal(qc.col, qo.col)
    assert np.array_equal(qc.val, qo.val) and np.array_equal(qc.lin, qo.lin)
    R = 128
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_BF16)
    c0 = oracle_c0(qo)
    x0, y0 = inputs.random_state(qo.n, R, 91, 0.9)
    J, h, _ = _oracle_J(qo, sb.SB_J_BF16)
    rows = np.random.default_rng(1).choice(qo.n, 300, replace=False)
    x64, y64 = x0.astype(np.float64), y0.astype(np.float64)
    a_k = float(np.float32(0.55))
    for variant, rpc in (("bsb", 0), ("bsb", 32), ("dsb", 0), ("dsb", 32)):
        sb.sb_set_option(ctx, sb.SB_OPT_STEP_RPC, rpc)
        sb.sb_set_state(ctx, x0, y0)
        sb.sb_advance(ctx, variant, 1.0, c0, 0.5, 1, _sched([0.55]))
        xg, yg = sb.sb_get_state(ctx)
        v = {"bsb": osb.BSB, "dsb": osb.DSB}[variant]
        xo, yo = osb.step_rows(J, h, x64, y64, rows, a_k, 1.0, c0, 0.5, v)
        xpre = osb.prewall_x(J, h, x64, y64, a_k, 1.0, c0, 0.5, v, rows=rows)
        compare_step(xg[rows], yg[rows], xo, yo, xpre)
    sb.sb_destroy(ctx)


def test_full_size_batch512_sampled_events():
    B = BATCH512
    tracks = batch512_tracks()
    p = sb.build_params(**B["cuts"])

    def build(e):
        ev = sb.sb_event_generate(B["seed0"] + e, sb.event_params(n_tracks=tracks[e],
                                                                  noise_frac=B["noise_frac"]))
        return sb.sb_qubo_build(ev, p)

    with ThreadPoolExecutor(max_workers=16) as ex:
        qs = list(ex.map(build, range(B["n_events"])))
    R = B["replicas"]
    NS = sum(q.n for q in qs)
    ctx = sb.sb_create_batch([(q.rowptr, q.col, q.val, q.lin) for q in qs], sb.SB_J_BF16)
    sb.sb_run(ctx, "dsb", B["a0"], 0.0, B["dt"], 0, R, seed=5)
    xi, _ = sb.sb_get_state(ctx)
    x0, y0 = inputs.random_state(NS, R, 93, 0.9)
    sb.sb_set_state(ctx, x0, y0)
    a_k = float(np.float32(0.45))
    sb.sb_advance(ctx, "dsb", B["a0"], 0.0, B["dt"], 1, _sched([0.45]))
    x, y = sb.sb_get_state(ctx)
    row0 = np.concatenate([[0], np.cumsum([q.n for q in qs])])
    small = [e for e in range(B["n_events"]) if tracks[e] <= 200]
    picks = [small[0], small[len(small) // 2], small[-1]]
    for e in picks:
        ev_o = oev.generate(B["seed0"] + e, oev.EventParams(n_tracks=tracks[e],
                                                           noise_frac=B["noise_frac"]))
        qo = oq.build_qubo(ev_o, oracle_params(B["cuts"]))
        q = qs[e]
        assert np.array_equal(q.col, qo.col) and np.array_equal(q.val, qo.val)
        J, h, _ = _oracle_J(qo, sb.SB_J_BF16)
        c0 = ising.c0_auto(ising.to_ising(qo)[0], qo.n)
        assert sb.sb_info(ctx, e)["c0_auto"] == pytest.approx(c0, rel=1e-12)
        c0 = float(np.float32(c0))
        sl = slice(int(row0[e]), int(row0[e + 1]))
        xs, _ = osb.init_state(5, qo.n, R, event=e)
        assert np.array_equal(xi[sl].astype(np.float64), xs), e
        xp, yp = x0[sl].astype(np.float64), y0[sl].astype(np.float64)
        xo, yo = osb.step(J, h, xp, yp, a_k, B["a0"], c0, B["dt"], osb.DSB)
        xpre = osb.prewall_x(J, h, xp, yp, a_k, B["a0"], c0, B["dt"], osb.DSB)
        compare_step(x[sl], y[sl], xo, yo, xpre)
    sb.sb_destroy(ctx)


def test_full_size_batch512_factored_dsb_step():
    """The bench's configuration: the 512-event batch with the shared-hit factor
    (hit ids offset per event), R = 64, dSB with sign bytes. One step from a
    random full-size state equals the plain sign-byte kernel's bit for bit over
    every event (all partial sums are exact multiples of 1/4), and sampled
    events, up to a 1000-track one, match the oracle run of that event alone."""
    B = BATCH512
    tracks = batch512_tracks()
    p = sb.build_params(**B["cuts"])

    def build(e):
        ev = sb.sb_event_generate(B["seed0"] + e, sb.event_params(n_tracks=tracks[e],
                                                                  noise_frac=B["noise_frac"]))
        return sb.sb_qubo_build(ev, p)

    with ThreadPoolExecutor(max_workers=16) as ex:
        qs = list(ex.map(build, range(B["n_events"])))
    R = B["replicas"]
    NS = sum(q.n for q in qs)
    off, mems = 0, []
    for q in qs:
        m, couple, wc, n_ids = sb.sb_qubo_factor(q)
        mems.append(np.where(m >= 0, m + off, -1))
        off += n_ids
    x0, y0 = inputs.random_state(NS, R, 97, 0.9)
    outs = []
    for factor in (True, False):
        ctx = sb.sb_create_batch([(q.rowptr, q.col, q.val, q.lin) for q in qs], sb.SB_J_BF16)
        if factor:
            sb.sb_set_factor(ctx, off, np.concatenate(mems), couple, wc)
            assert sb.sb_factor_info(ctx)["rows"] > NS // 2
        sb.sb_set_state(ctx, x0, y0)
        sb.sb_advance(ctx, "dsb", B["a0"], 0.0, B["dt"], 1, _sched([0.45]))
        outs.append(sb.sb_get_state(ctx))
        if factor:
            infos = [sb.sb_info(ctx, e) for e in range(len(qs))]
        sb.sb_destroy(ctx)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    x, y = outs[0]
    a_k = float(np.float32(0.45))
    row0 = np.concatenate([[0], np.cumsum([q.n for q in qs])])
    order = np.argsort(tracks, kind="stable")
    picks = [int(order[50]), int(order[256]), int(np.argmin(np.abs(np.asarray(tracks) - 1000)))]
    for e in picks:
        ev_o = oev.generate(B["seed0"] + e, oev.EventParams(n_tracks=tracks[e],
                                                           noise_frac=B["noise_frac"]))
        qo = oq.build_qubo(ev_o, oracle_params(B["cuts"]))
        assert np.array_equal(qs[e].col, qo.col) and np.array_equal(qs[e].val, qo.val)
        J, h, _ = _oracle_J(qo, sb.SB_J_BF16)
        c0 = ising.c0_auto(ising.to_ising(qo)[0], qo.n)
        assert infos[e]["c0_auto"] == pytest.approx(c0, rel=1e-12)
        c0 = float(np.float32(c0))
        sl = slice(int(row0[e]), int(row0[e + 1]))
        xp, yp = x0[sl].astype(np.float64), y0[sl].astype(np.float64)
        xo, yo = osb.step(J, h, xp, yp, a_k, B["a0"], c0, B["dt"], osb.DSB)
        xpre = osb.prewall_x(J, h, xp, yp, a_k, B["a0"], c0, B["dt"], osb.DSB)
        compare_step(x[sl], y[sl], xo, yo, xpre)
