"""GPU path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 energies of a given spin vector 1e-12 relative; one FP32 SB
step 1e-5 (max error over the state normalised by the state's max |value|);
initial state, CSR handling, arg-min and selections bit-exact."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from oracle import ising, sb as osb, tracks as otr
from tests import inputs
from tests.gpu_common import (compare_step, compare_step_elementwise, max_rel, oracle_c0,
                              workload_qubos)

pytestmark = pytest.mark.gpu
VARIANTS = [osb.ASB, osb.BSB, osb.DSB]


def _ctx(q, prec=sb.SB_J_FP32):
    return sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, prec)


def _sched(vals):
    return torch.tensor(np.asarray(vals, np.float32), device="cuda")


def _bf16_round(v):
    return torch.tensor(v, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()


def _oracle_J(q, prec):
    J, h, off = ising.to_ising(q)
    if prec == sb.SB_J_BF16:
        J = J.copy()
        J.data = _bf16_round(J.data)
    return J, h, off


# ------------------------------------------------------------------ conversion / energies
@pytest.mark.parametrize("name", ["event100", "event1000"])
def test_ising_scalars_match_oracle(name):
    _, qc, _, qo = workload_qubos(name)
    ctx = _ctx(qc)
    info = sb.sb_info(ctx)
    J, h, off = ising.to_ising(qo)
    assert info["n"] == qo.n and info["nnz"] == len(qo.col)
    assert info["offset"] == pytest.approx(off, rel=1e-12, abs=1e-12)
    assert info["sigma_j"] == pytest.approx(ising.sigma_j(J, qo.n), rel=1e-12)
    assert info["c0_auto"] == pytest.approx(ising.c0_auto(J, qo.n), rel=1e-12)


@pytest.mark.parametrize("name,R", [("event100", 1), ("event100", 7), ("event1000", 16)])
def test_energy_of_given_spins(name, R):
    _, qc, _, qo = workload_qubos(name)
    ctx = _ctx(qc)
    T = inputs.random_spins(qo.n, R, seed=R)
    spins = np.where(T > 0, 1, -1).astype(np.int8)
    E_gpu = sb.sb_energy(ctx, spins)[0]
    E_orc = ising.qubo_energy(qo, T)
    np.testing.assert_allclose(E_gpu, E_orc, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(E_orc).max()))
    # the Ising form with the offset gives the same numbers
    J, h, off = ising.to_ising(qo)
    np.testing.assert_allclose(E_gpu, ising.ising_energy(J, h, 2.0 * T - 1.0) + off, rtol=1e-12,
                               atol=1e-10)


def test_energy_edge_cases():
    # all zeros -> 0, all ones -> sum a + sum_{i<j} b
    _, qc, _, qo = workload_qubos("event100")
    ctx = _ctx(qc)
    for fill in (0, 1):
        T = np.full((qo.n, 3), fill, np.int8)
        E = sb.sb_energy(ctx, np.where(T > 0, 1, -1).astype(np.int8))[0]
        np.testing.assert_allclose(E, ising.qubo_energy(qo, T), rtol=1e-12, atol=1e-12)
    # a single variable without couplings
    ctx1 = sb.sb_create(1, np.array([0, 0]), np.zeros(0), np.zeros(0), np.array([-0.5]))
    assert sb.sb_energy(ctx1, np.array([[1, -1]], np.int8))[0].tolist() == [-0.5, 0.0]


# ------------------------------------------------------------------ initial state
@pytest.mark.parametrize("R", [1, 3, 64, 256])
def test_initial_state_bit_exact(R):
    _, qc, _, qo = workload_qubos("event100")
    ctx = _ctx(qc)
    sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 0, R, seed=12345)
    xg, yg = sb.sb_get_state(ctx)
    xo, yo = osb.init_state(12345, qo.n, R)
    assert np.array_equal(xg.astype(np.float64), xo)
    assert np.array_equal(yg.astype(np.float64), yo)


# ------------------------------------------------------------------ one SB step
def _one_step_case(q, qo, prec, variant, R, seed, a_k, scale, graph=False):
    ctx = _ctx(q, prec)
    if not graph:
        sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    c0 = oracle_c0(qo)
    x0, y0 = inputs.random_state(qo.n, R, seed, scale)
    sb.sb_set_state(ctx, x0, y0)
    sb.sb_advance(ctx, variant, 1.0, c0, 0.5, 1, _sched([a_k]))
    xg, yg = sb.sb_get_state(ctx)
    J, h, _ = _oracle_J(qo, prec)
    a32 = float(np.float32(a_k))
    xo, yo = osb.step(J, h, x0.astype(np.float64), y0.astype(np.float64), a32, 1.0, c0, 0.5, variant)
    xpre = osb.prewall_x(J, h, x0.astype(np.float64), y0.astype(np.float64), a32, 1.0, c0, 0.5, variant)
    compare_step_elementwise(J, h, x0, y0, a32, 1.0, c0, 0.5, variant, xg, yg, xo, yo, xpre)
    return compare_step(xg, yg, xo, yo, xpre)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("R", [1, 3, 32, 64, 256])
def test_one_step_fp32(variant, R):
    _, qc, _, qo = workload_qubos("event100")
    _one_step_case(qc, qo, sb.SB_J_FP32, variant, R, seed=R + 10 * variant, a_k=0.37, scale=0.8)


@pytest.mark.parametrize("variant", VARIANTS)
def test_one_step_bf16(variant):
    _, qc, _, qo = workload_qubos("event100")
    _one_step_case(qc, qo, sb.SB_J_BF16, variant, 32, seed=5, a_k=0.81, scale=1.0)


def test_one_step_random_weights_bf16_quantised():
    """Couplings that BF16 does not represent exactly: the oracle is fed the
    BF16-rounded J so the step comparison isolates the arithmetic."""
    q = inputs.random_qubo(300, 12, seed=2, values=(-0.731, 0.377, 1.234), lin_low=-1, lin_high=1)
    for variant in VARIANTS:
        _one_step_case(q, q, sb.SB_J_BF16, variant, 8, seed=variant, a_k=0.5, scale=1.0)
        _one_step_case(q, q, sb.SB_J_FP32, variant, 5, seed=variant, a_k=0.5, scale=1.0)


@pytest.mark.parametrize("variant", VARIANTS)
def test_short_horizon_from_seeded_start(variant):
    """20 steps from the Philox start on the linear schedule: the GPU trajectory
    against the free-running oracle (each side draws the start itself), and
    single steps from states along the oracle's own trajectory (rounded to FP32
    and given to both sides). aSB has no wall: its x^3 force makes explicit
    steps of dt = 0.5 blow up within a few steps (FP32 overflows first), so it
    runs with dt = 0.1."""
    _, qc, _, qo = workload_qubos("event100")
    R, S = 16, 20
    dt = 0.1 if variant == osb.ASB else 0.5
    ctx = _ctx(qc)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    c0 = oracle_c0(qo)
    sched = np.float32(np.linspace(0.0, 1.0, 2000))[:S]
    J, h, _ = ising.to_ising(qo)
    # free-running trajectories
    sb.sb_run(ctx, variant, 1.0, c0, dt, 0, R, seed=99)
    sb.sb_advance(ctx, variant, 1.0, c0, dt, S, _sched(sched))
    xg, yg = sb.sb_get_state(ctx)
    assert np.all(np.isfinite(xg)) and np.all(np.isfinite(yg))
    xf, yf = osb.init_state(99, qo.n, R)
    states = {}
    for k in range(S):
        if k in (0, 5, 10, 19):
            states[k] = (xf.astype(np.float32), yf.astype(np.float32))
        xf, yf = osb.step(J, h, xf, yf, float(sched[k]), 1.0, c0, dt, variant)
    assert max_rel(xg, xf) < 1e-4 and max_rel(yg, yf) < 1e-4
    # single steps from oracle states
    for k, (x32, y32) in states.items():
        sb.sb_set_state(ctx, x32, y32)
        sb.sb_advance(ctx, variant, 1.0, c0, dt, 1, _sched(sched[k:k + 1]))
        xn, yn = sb.sb_get_state(ctx)
        xp, yp = x32.astype(np.float64), y32.astype(np.float64)
        xo, yo = osb.step(J, h, xp, yp, float(sched[k]), 1.0, c0, dt, variant)
        xpre = osb.prewall_x(J, h, xp, yp, float(sched[k]), 1.0, c0, dt, variant)
        compare_step(xn, yn, xo, yo, xpre)


def test_graph_and_direct_launches_agree_bit_for_bit():
    """With graphs on, a run shape is launched directly the first time, captured
    the second time it repeats and replayed after that: all agree with direct
    launches bit for bit."""
    _, qc, _, qo = workload_qubos("event100")
    ref = _ctx(qc, sb.SB_J_BF16)
    sb.sb_set_option(ref, sb.SB_OPT_GRAPH, 0)
    sb.sb_run(ref, "dsb", 1.0, 0.0, 0.5, 37, 8, seed=4)
    xr, yr = sb.sb_get_state(ref)
    ctx = _ctx(qc, sb.SB_J_BF16)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 1)
    for _ in range(3):   # direct, capture, replay
        sb.sb_run(ctx, "dsb", 1.0, 0.0, 0.5, 37, 8, seed=4)
        x, y = sb.sb_get_state(ctx)
        assert np.array_equal(x, xr) and np.array_equal(y, yr)


def test_wall_invariant_and_empty_rows():
    # an isolated variable (empty CSR row) next to coupled ones
    q = inputs.random_qubo(50, 3, seed=8)
    rp = np.concatenate([q.rowptr, [q.rowptr[-1]]]).astype(np.int32)
    lin = np.concatenate([q.lin, [-0.3]])
    ctx = sb.sb_create(51, rp, q.col, q.val, lin)
    for v in ("bsb", "dsb"):
        sb.sb_run(ctx, v, 1.0, 0.0, 0.5, 300, 5, seed=1)
        x, y = sb.sb_get_state(ctx)
        assert np.all(np.abs(x) <= 1.0)
        assert np.all(y[np.abs(x) == 1.0] == 0.0)


# ------------------------------------------------------------------ full-size sampled checks
def test_full_size_event1000_step_sampled():
    """The bench workload (1000 tracks, R = 256, BF16 J, graph replay): one step
    from a random full-size state, 300 sampled rows checked against the oracle."""
    _, qc, _, qo = workload_qubos("event1000")
    R = 256
    ctx = _ctx(qc, sb.SB_J_BF16)
    c0 = oracle_c0(qo)
    x0, y0 = inputs.random_state(qo.n, R, 77, 0.9)
    J, h, _ = _oracle_J(qo, sb.SB_J_BF16)
    rows = np.random.default_rng(0).choice(qo.n, 300, replace=False)
    for variant in VARIANTS:
        sb.sb_set_state(ctx, x0, y0)
        sched = _sched(np.full(8, 0.6, np.float32))
        sb.sb_advance(ctx, variant, 1.0, c0, 0.5, 1, sched)
        xg, yg = sb.sb_get_state(ctx)
        xo, yo = osb.step_rows(J, h, x0.astype(np.float64), y0.astype(np.float64), rows,
                               float(np.float32(0.6)), 1.0, c0, 0.5, variant)
        xpre = osb.prewall_x(J, h, x0.astype(np.float64), y0.astype(np.float64),
                             float(np.float32(0.6)), 1.0, c0, 0.5, variant, rows=rows)
        compare_step(xg[rows], yg[rows], xo, yo, xpre)


def test_full_size_event1000_readout():
    """Readout at the bench shape (R = 256, BF16 J) of a seeded full-size state:
    energies of sampled replicas against the oracle, and the arg-min and the best
    selection consistent with them."""
    _, qc, _, qo = workload_qubos("event1000")
    R = 256
    ctx = _ctx(qc, sb.SB_J_BF16)
    x0, y0 = inputs.random_state(qo.n, R, 123, 1.0)
    sb.sb_set_state(ctx, x0, y0)
    T, Ebest, rbest = sb.sb_best(ctx)
    E_all = sb.sb_energy(ctx, None, R)[0]
    Ts = (x0 > 0).astype(np.int8)
    pick = [0, 17, int(rbest[0]), R - 1]
    np.testing.assert_allclose(E_all[pick], ising.qubo_energy(qo, Ts[:, pick]), rtol=1e-12)
    assert int(rbest[0]) == int(np.argmin(E_all))
    assert Ebest[0] == E_all[rbest[0]]
    assert np.array_equal(T, Ts[:, rbest[0]].astype(np.uint8))


# ------------------------------------------------------------------ statistics over seeds
@pytest.mark.parametrize("variant", [osb.BSB, osb.DSB])
def test_final_energy_statistics_64_replicas(variant):
    """event100, 2000 steps: over 64 independent starts the median final QUBO
    energy of the GPU is within 0.5 % of the oracle's, and the efficiency /
    purity of the best run within one point."""
    ev_c, qc, ev_o, qo = workload_qubos("event100")
    R, S = 64, 2000
    ctx = _ctx(qc)
    c0 = oracle_c0(qo)
    sb.sb_run(ctx, variant, 1.0, c0, 0.5, S, R, seed=2024)
    E_gpu = sb.sb_energy(ctx, None, R)[0]
    J, h, _ = ising.to_ising(qo)
    x, y = osb.init_state(2024, qo.n, R)
    res = osb.run(J, h, x, y, osb.linear_schedule(1.0, S), 1.0, c0, 0.5, variant)
    T_o = ising.triplets_from_spins(ising.spins_from_x(res.x))
    E_orc = ising.qubo_energy(qo, T_o)
    med_g, med_o = float(np.median(E_gpu)), float(np.median(E_orc))
    assert abs(med_g - med_o) <= 0.005 * abs(med_o)
    T_g, _, _ = sb.sb_best(ctx)
    sc_g = sb.sb_tracks(ev_c, qc, T_g)
    _, reco = otr.assemble(qo, T_o[:, int(np.argmin(E_orc))])
    _, _, _, eff_o, pur_o = otr.score(ev_o, reco)
    assert abs(sc_g["efficiency"] - eff_o) <= 0.01
    assert abs(sc_g["purity"] - pur_o) <= 0.01


# ------------------------------------------------------------------ batched events
def test_batch_matches_oracle_per_event():
    """Three events in one context: each event's initial state, one step and
    energies agree with the oracle run on that event alone."""
    qs = [inputs.random_qubo(n, 6, seed=n) for n in (40, 130, 7)]
    ctx = sb.sb_create_batch([(q.rowptr, q.col, q.val, q.lin) for q in qs])
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    R = 12
    sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 0, R, seed=31)
    x0, y0 = sb.sb_get_state(ctx)
    sb.sb_advance(ctx, "bsb", 1.0, 0.0, 0.5, 1, _sched([0.4]))
    x1, y1 = sb.sb_get_state(ctx)
    spins = inputs.random_spins(sum(q.n for q in qs), R, seed=6)
    E = sb.sb_energy(ctx, np.where(spins > 0, 1, -1).astype(np.int8))
    row0 = 0
    for e, q in enumerate(qs):
        sl = slice(row0, row0 + q.n)
        xo, yo = osb.init_state(31, q.n, R, event=e)
        assert np.array_equal(x0[sl].astype(np.float64), xo)
        J, h, _ = ising.to_ising(q)
        c0 = ising.c0_auto(J, q.n)
        assert sb.sb_info(ctx, e)["c0_auto"] == pytest.approx(c0, rel=1e-12)
        xn, yn = osb.step(J, h, xo, yo, float(np.float32(0.4)), 1.0, c0, 0.5, osb.BSB)
        assert max_rel(x1[sl], xn) < 1e-5 and max_rel(y1[sl], yn) < 1e-5
        np.testing.assert_allclose(E[e], ising.qubo_energy(q, spins[sl]), rtol=1e-12, atol=1e-12)
        row0 += q.n


@pytest.mark.parametrize("variant", ["asb", "bsb", "dsb"])
@pytest.mark.parametrize("prec", [sb.SB_J_FP32, sb.SB_J_BF16])
@pytest.mark.parametrize("R", [32, 96, 256])
def test_tiled_and_untiled_kernels_bit_identical(variant, prec, R):
    """The row-block tiled step and the untiled step run the same FMA sequence
    per (row, replica): their states must agree bit for bit."""
    _, qc, _, _ = workload_qubos("event500")
    dt = 0.1 if variant == "asb" else 0.5
    out = []
    for tiled in (1, 0):
        ctx = _ctx(qc, prec)
        sb.sb_set_option(ctx, sb.SB_OPT_TILED, tiled)
        sb.sb_run(ctx, variant, 1.0, 0.0, dt, 25, R, seed=R)
        out.append(sb.sb_get_state(ctx))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_batch_tiled_matches_single_events():
    """A batch of two events with R = 32 (tiled kernel; row blocks may straddle
    the event boundary) gives each event, from the same starting state, the
    bit-identical trajectory of its own single-event context."""
    qs = [workload_qubos("event100")[1], inputs.random_qubo(300, 9, seed=3)]
    R, S = 32, 30
    ctxb = sb.sb_create_batch([(q.rowptr, q.col, q.val, q.lin) for q in qs])
    singles = [_ctx(q) for q in qs]
    states = [inputs.random_state(q.n, R, 40 + k, 0.5) for k, q in enumerate(qs)]
    sb.sb_set_state(ctxb, np.concatenate([s[0] for s in states]),
                    np.concatenate([s[1] for s in states]))
    sched = _sched(np.float32(np.linspace(0, 1, S)))
    sb.sb_advance(ctxb, "dsb", 1.0, 0.0, 0.5, S, sched)
    xb, yb = sb.sb_get_state(ctxb)
    row0 = 0
    for q, ctx, (x0, y0) in zip(qs, singles, states):
        sb.sb_set_state(ctx, x0, y0)
        sb.sb_advance(ctx, "dsb", 1.0, 0.0, 0.5, S, sched)
        x, y = sb.sb_get_state(ctx)
        assert np.array_equal(xb[row0:row0 + q.n], x) and np.array_equal(yb[row0:row0 + q.n], y)
        row0 += q.n


@pytest.mark.parametrize("R", [64, 256])
def test_autotune_keeps_results_and_picks_a_valid_config(R):
    _, qc, _, _ = workload_qubos("event500")
    ref = _ctx(qc, sb.SB_J_BF16)
    sb.sb_run(ref, "bsb", 1.0, 0.0, 0.5, 20, R, seed=5)
    x_ref, y_ref = sb.sb_get_state(ref)
    ctx = _ctx(qc, sb.SB_J_BF16)
    cfg, us = sb.sb_autotune(ctx, "bsb", R, trial_steps=10)
    assert cfg["tiled"] in (0, 1) and cfg["rows_per_warp"] in (0, 2, 4) and us > 0
    sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 20, R, seed=5)
    x, y = sb.sb_get_state(ctx)
    assert np.array_equal(x, x_ref) and np.array_equal(y, y_ref)


@pytest.mark.parametrize("rt,rpc", [(32, 0), (64, 96), (128, 40), (0, 512)])
def test_step_tiling_options_bit_identical(rt, rpc):
    _, qc, _, _ = workload_qubos("event500")
    out = []
    for opts in ((0, 0), (rt, rpc)):
        ctx = _ctx(qc)
        sb.sb_set_option(ctx, 2, opts[0])
        sb.sb_set_option(ctx, 3, opts[1])
        sb.sb_run(ctx, "dsb", 1.0, 0.0, 0.5, 15, 128, seed=2)
        out.append(sb.sb_get_state(ctx))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("R", [1, 3, 64, 256])
def test_dsb_sign_gather_bit_identical(R):
    """dSB gathering int8 signs gives the state of dSB gathering FP32 positions,
    also across sb_set_state / sb_advance boundaries and graph replay."""
    _, qc, _, _ = workload_qubos("event500")
    out = []
    for signs in (1, 0):
        ctx = _ctx(qc, sb.SB_J_BF16)
        sb.sb_set_option(ctx, 5, signs)
        sb.sb_run(ctx, "dsb", 1.0, 0.0, 0.5, 12, R, seed=R + 1)
        x, y = sb.sb_get_state(ctx)
        sb.sb_set_state(ctx, x, y)
        sb.sb_advance(ctx, "dsb", 1.0, 0.0, 0.5, 9, _sched(np.float32(np.linspace(0.2, 0.9, 9))))
        out.append(sb.sb_get_state(ctx))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("variant", ["bsb", "dsb"])
@pytest.mark.parametrize("unroll,rpc", [(4, -1), (4, 32)])
def test_unroll_and_wave_options_bit_identical(variant, unroll, rpc):
    _, qc, _, _ = workload_qubos("event500")
    out = []
    for opts in ((4, 0), (unroll, rpc)):
        ctx = _ctx(qc, sb.SB_J_BF16)
        sb.sb_set_option(ctx, 4, opts[0])
        sb.sb_set_option(ctx, 3, opts[1])
        sb.sb_run(ctx, variant, 1.0, 0.0, 0.5, 20, 256, seed=4)
        out.append(sb.sb_get_state(ctx))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


# ------------------------------------------------------------------ paper-exact weights (Eq. 14, 15)
def _paper_qubos():
    from paper_2402_14718_gb300.workloads import CUTS_S8
    from oracle import events as oev, qubo as oq
    kw = dict(CUTS_S8, coupling_mode=1, bias_mode=1)
    ev_c = sb.sb_event_generate(0, sb.event_params(n_tracks=100))
    qc = sb.sb_qubo_build(ev_c, sb.build_params(**kw))
    kw["five_hit_rule"] = True
    qo = oq.build_qubo(oev.generate(0, oev.EventParams(n_tracks=100)), oq.BuildParams(**kw))
    return qc, qo


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", [sb.SB_J_FP32, sb.SB_J_BF16])
def test_paper_weights_one_step(variant, prec):
    qc, qo = _paper_qubos()
    _one_step_case(qc, qo, prec, variant, 32, seed=13 + variant, a_k=0.45, scale=0.9)


def test_paper_weights_bf16_quantisation_effect():
    """-S_ij / 4 is not exact in BF16 (8 significant bits, round to nearest): the
    J error is at most 2^-8 relative, and over a full 2000-step bSB run the
    median final energy of 64 replicas moves by less than 0.5 %."""
    qc, _ = _paper_qubos()
    J = -qc.val / 4.0
    Jb = _bf16_round(J)
    rel = np.max(np.abs(Jb - J) / np.abs(J))
    assert 0.0 < rel <= 2.0 ** -8
    med = []
    for prec in (sb.SB_J_FP32, sb.SB_J_BF16):
        ctx = _ctx(qc, prec)
        sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 2000, 64, seed=77)
        med.append(float(np.median(sb.sb_energy(ctx, None, 64)[0])))
    assert abs(med[1] - med[0]) <= 0.005 * abs(med[0])



@pytest.mark.parametrize("variant", ["asb", "bsb", "dsb"])
def test_single_replica_kernel_bit_identical(variant):
    """R = 1 runs on a dedicated one-thread-per-row kernel; forcing the generic
    kernel (rows-per-CTA override) gives the same state bit for bit."""
    _, qc, _, _ = workload_qubos("event500")
    dt = 0.1 if variant == "asb" else 0.5
    out = []
    for rpc in (0, 300):
        ctx = _ctx(qc)
        sb.sb_set_option(ctx, 3, rpc)
        sb.sb_run(ctx, variant, 1.0, 0.0, dt, 40, 1, seed=9)
        out.append(sb.sb_get_state(ctx))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])



@pytest.mark.parametrize("variant", ["bsb", "dsb"])
@pytest.mark.parametrize("groups,R", [(2, 256), (4, 256), (2, 64)])
def test_sequential_replica_groups_bit_identical(variant, groups, R):
    _, qc, _, _ = workload_qubos("event500")
    out = []
    for g in (1, groups):
        ctx = _ctx(qc, sb.SB_J_BF16)
        sb.sb_set_option(ctx, 6, g)
        sb.sb_run(ctx, variant, 1.0, 0.0, 0.5, 21, R, seed=3)
        out.append(sb.sb_get_state(ctx))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])



def test_l2_persist_option_bit_identical():
    _, qc, _, _ = workload_qubos("event500")
    out = []
    for l2 in (0, 1):
        for graph in (0, 1):
            ctx = _ctx(qc, sb.SB_J_BF16)
            sb.sb_set_option(ctx, 7, l2)
            sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, graph)
            sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 16, 64, seed=6)
            out.append(sb.sb_get_state(ctx))
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0]) and np.array_equal(o[1], out[0][1])


@pytest.mark.parametrize("lanes", [8, 16, 32])
@pytest.mark.parametrize("variant", ["asb", "bsb", "dsb"])
def test_one_replica_lane_groups_bit_identical(lanes, variant):
    """SB_OPT_R1_LANES: G lanes per row gather in parallel and form the same
    CSR-order FMA chain as the one-thread-per-row kernel (R = 1): equal states
    for FP32 and BF16 J, graph replay and direct launches, a batched context."""
    _, qc, _, _ = workload_qubos("event1000")
    qs = [workload_qubos("event100")[1], qc]
    dt = 0.1 if variant == "asb" else 0.5
    for prec in (sb.SB_J_FP32, sb.SB_J_BF16):
        for graph in (1, 0):
            outs = []
            for r1 in (lanes, 0):
                ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, prec)
                sb.sb_set_option(ctx, sb.SB_OPT_R1_LANES, r1)
                sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, graph)
                sb.sb_run(ctx, variant, 1.0, 0.0, dt, 60, 1, seed=2)
                sb.sb_run(ctx, variant, 1.0, 0.0, dt, 60, 1, seed=2)
                outs.append(sb.sb_get_state(ctx))
                sb.sb_destroy(ctx)
            assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    outs = []
    for r1 in (lanes, 0):
        ctxb = sb.sb_create_batch([(q.rowptr, q.col, q.val, q.lin) for q in qs])
        sb.sb_set_option(ctxb, sb.SB_OPT_R1_LANES, r1)
        sb.sb_run(ctxb, variant, 1.0, 0.0, dt, 40, 1, seed=3)
        outs.append(sb.sb_get_state(ctxb))
        sb.sb_destroy(ctxb)
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
