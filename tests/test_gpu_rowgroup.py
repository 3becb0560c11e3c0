"""Row-group step kernel (SB_OPT_ROWS_PER_WARP): a warp owns a group of 2 or
4 rows that share neighbours and loads each union column once for all of them.

Each (row, replica) still takes one FMA per nonzero in CSR order, so the
states must equal the untiled kernel's bit for bit; one step is also checked
against the FP64 oracle (1e-5)."""
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


def _run(q, prec, variant, R, steps, rw, seed=3, graph=1, rt=0, rpc=0, state=None, heavy=1):
    ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, prec)
    sb.sb_set_option(ctx, sb.SB_OPT_ROWS_PER_WARP, rw)
    sb.sb_set_option(ctx, sb.SB_OPT_HEAVY_FIRST, heavy)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, graph)
    sb.sb_set_option(ctx, sb.SB_OPT_STEP_RT, rt)
    sb.sb_set_option(ctx, sb.SB_OPT_STEP_RPC, rpc)
    dt = 0.1 if variant == "asb" else 0.5
    if state is None:
        sb.sb_run(ctx, variant, 1.0, 0.0, dt, steps, R, seed=seed)
    else:
        sb.sb_set_state(ctx, *state)
        sb.sb_advance(ctx, variant, 1.0, 0.0, dt, steps, _sched(np.linspace(0, 1, steps)))
    x, y = sb.sb_get_state(ctx)
    return ctx, x, y


def _same(q, prec, variant, R, steps, rw, **kw):
    _, xg, yg = _run(q, prec, variant, R, steps, rw, **kw)
    kw.pop("rt", None)
    kw.pop("rpc", None)
    kw.pop("heavy", None)
    _, xu, yu = _run(q, prec, variant, R, steps, 0, **kw)
    assert np.array_equal(xg, xu) and np.array_equal(yg, yu)


@pytest.mark.parametrize("rw", [2, 4])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", [sb.SB_J_FP32, sb.SB_J_BF16])
@pytest.mark.parametrize("R", [128, 256, 384, 64])
def test_rowgroup_and_untiled_bit_identical(rw, variant, prec, R):
    """R = 128 / 384 use 128-replica warps, 256 one 256-replica warp per group;
    R = 64 is not a multiple of 128 and falls back to the untiled kernel."""
    _, qc, _, _ = workload_qubos("event500")
    _same(qc, prec, variant, R, 25, rw)


@pytest.mark.parametrize("rpc", [0, 32, 64])
@pytest.mark.parametrize("variant", VARIANTS)
def test_rowgroup_row_order_dispatch(rpc, variant):
    """SB_OPT_HEAVY_FIRST = 0 (CTAs in row order) against the untiled kernel;
    the heavy-first order is covered by every other row-group test (and, for
    the dSB sign-byte kernel, by the automatic choice on these sizes)."""
    _, qc, _, _ = workload_qubos("event500")
    _same(qc, sb.SB_J_BF16, variant, 256, 15, 2, rpc=rpc, heavy=0)
    _same(qc, sb.SB_J_FP32, variant, 128, 15, 4, rpc=rpc, heavy=0)
    if variant == "dsb":   # the sign-byte kernel: row order against the default order
        _same(qc, sb.SB_J_BF16, variant, 256, 15, 0, rpc=rpc, heavy=0)


def test_heavy_first_option_range_and_auto():
    """-1 (default) picks the order from the L2 fit; the states are the same
    under every order."""
    _, qc, _, _ = workload_qubos("event500")
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin)
    with pytest.raises(sb.SbError):
        sb.sb_set_option(ctx, sb.SB_OPT_HEAVY_FIRST, 2)
    sb.sb_destroy(ctx)
    _same(qc, sb.SB_J_BF16, "bsb", 256, 15, 2, heavy=-1)


@pytest.mark.parametrize("rt,rpc", [(128, 0), (0, 32), (128, 64), (0, -1)])
def test_rowgroup_tile_and_chunk_options(rt, rpc):
    _, qc, _, _ = workload_qubos("event500")
    for rw in (2, 4):
        _same(qc, sb.SB_J_BF16, "bsb", 256, 12, rw, rt=rt, rpc=rpc)


@pytest.mark.parametrize("variant", VARIANTS)
def test_rowgroup_one_step_against_oracle(variant):
    _, qc, _, qo = workload_qubos("event100")
    R = 128
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_FP32)
    sb.sb_set_option(ctx, sb.SB_OPT_ROWS_PER_WARP, 4)
    sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
    c0 = oracle_c0(qo)
    x0, y0 = inputs.random_state(qo.n, R, 21 + len(variant), 0.8)
    sb.sb_set_state(ctx, x0, y0)
    a_k = 0.61
    sb.sb_advance(ctx, variant, 1.0, c0, 0.5, 1, _sched([a_k]))
    xg, yg = sb.sb_get_state(ctx)
    J, h, _ = _oracle_J(qo, sb.SB_J_FP32)
    v = {"asb": osb.ASB, "bsb": osb.BSB, "dsb": osb.DSB}[variant]
    a32 = float(np.float32(a_k))
    x64, y64 = x0.astype(np.float64), y0.astype(np.float64)
    xo, yo = osb.step(J, h, x64, y64, a32, 1.0, c0, 0.5, v)
    xpre = osb.prewall_x(J, h, x64, y64, a32, 1.0, c0, 0.5, v)
    compare_step(xg, yg, xo, yo, xpre)


def test_rowgroup_ragged_sizes_empty_rows_and_dense_rows():
    """N not a multiple of the group size, isolated rows, rows of high degree,
    direct (non-graph) launches."""
    q = inputs.random_qubo(1000, 7, seed=31)
    rp = np.concatenate([q.rowptr, np.full(43, q.rowptr[-1])]).astype(np.int32)
    lin = np.concatenate([q.lin, np.linspace(-0.4, 0.4, 43)])
    qe = inputs.QuboArrays(1043, rp, q.col, q.val, lin)
    for rw in (2, 4):
        for variant in VARIANTS:
            _same(qe, sb.SB_J_FP32, variant, 128, 17, rw, graph=0)
        _same(qe, sb.SB_J_BF16, "dsb", 256, 9, rw)
    qd = inputs.random_qubo(401, 200, seed=5, values=(-1.0, 0.5, 2.0))
    _same(qd, sb.SB_J_FP32, "bsb", 256, 10, 4)
    qz = inputs.QuboArrays(70, np.zeros(71, np.int32), np.zeros(0, np.int32),
                           np.zeros(0), np.linspace(-1, 1, 70))
    _same(qz, sb.SB_J_FP32, "bsb", 128, 12, 2)


def test_rowgroup_batch_matches_single_events():
    """Row groups of a batched context may span two events (per-event c0)."""
    qs = [workload_qubos("event100")[1], inputs.random_qubo(301, 9, seed=3),
          inputs.random_qubo(77, 4, seed=4)]
    R, S = 128, 20
    states = [inputs.random_state(q.n, R, 60 + k, 0.5) for k, q in enumerate(qs)]
    ctxb = sb.sb_create_batch([(q.rowptr, q.col, q.val, q.lin) for q in qs])
    sb.sb_set_option(ctxb, sb.SB_OPT_ROWS_PER_WARP, 4)
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


def test_rowgroup_follows_weight_changes():
    """sb_set_weights rewrites J; the row-group entries are refilled from it."""
    _, qc, _, _ = workload_qubos("event500")
    out = []
    for rw in (4, 0):
        ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_BF16)
        sb.sb_set_option(ctx, sb.SB_OPT_ROWS_PER_WARP, rw)
        sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 3, 128, seed=1)   # builds the tables first
        sb.sb_set_weights(ctx, qc.cls, qc.quality, 0.7, 1.9)
        sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 15, 128, seed=2)
        out.append(sb.sb_get_state(ctx))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_rowgroup_full_size_event1000():
    """The 1000-track workload at R = 256 with BF16 J (the bench launch shape)."""
    _, qc, _, _ = workload_qubos("event1000")
    for rw in (2, 4):
        _same(qc, sb.SB_J_BF16, "bsb", 256, 8, rw, rpc=32)


@pytest.mark.parametrize("rw", [0, 2, 4])
@pytest.mark.parametrize("signs", [1, 0])
def test_dsb_exact_zero_and_wall_positions_against_oracle(rw, signs):
    """dSB uses sgn(x) with sgn(0) = 0. A state with exact zeros, exact +-1
    (walls) and ordinary values, one step, every dSB gather form (stored sign
    bytes or FP32 x, row groups or not) against the oracle, and the forms
    against each other bit for bit."""
    _, qc, _, qo = workload_qubos("event100")
    R = 128
    x0, y0 = inputs.random_state(qo.n, R, 77, 0.9)
    rng = np.random.default_rng(5)
    pick = rng.random(x0.shape)
    x0[pick < 0.2] = 0.0
    x0[(pick >= 0.2) & (pick < 0.4)] = 1.0
    x0[(pick >= 0.4) & (pick < 0.5)] = -1.0
    outs = []
    for form in ((rw, signs), (0, 0)):
        ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_FP32)
        sb.sb_set_option(ctx, sb.SB_OPT_ROWS_PER_WARP, form[0])
        sb.sb_set_option(ctx, sb.SB_OPT_DSB_SIGNS, form[1])
        sb.sb_set_option(ctx, sb.SB_OPT_GRAPH, 0)
        c0 = oracle_c0(qo)
        sb.sb_set_state(ctx, x0, y0)
        sb.sb_advance(ctx, "dsb", 1.0, c0, 0.5, 1, _sched([0.3]))
        outs.append(sb.sb_get_state(ctx))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    J, h, _ = _oracle_J(qo, sb.SB_J_FP32)
    a32 = float(np.float32(0.3))
    x64, y64 = x0.astype(np.float64), y0.astype(np.float64)
    xo, yo = osb.step(J, h, x64, y64, a32, 1.0, c0, 0.5, osb.DSB)
    xpre = osb.prewall_x(J, h, x64, y64, a32, 1.0, c0, 0.5, osb.DSB)
    compare_step(outs[0][0], outs[0][1], xo, yo, xpre)


def _with_huge_pairs(q, b_pair):
    """q plus a coupling b_pair between rows 2k and 2k + 1 (k = 0, 1, ...), with
    a_i - b_pair / 2 as the linear terms so that the field h stays small."""
    D = np.zeros((q.n, q.n))
    for i in range(q.n):
        D[i, q.col[q.rowptr[i]:q.rowptr[i + 1]]] = q.val[q.rowptr[i]:q.rowptr[i + 1]]
    for k in range(q.n // 2):
        D[2 * k, 2 * k + 1] = D[2 * k + 1, 2 * k] = b_pair
    rp = np.zeros(q.n + 1, np.int32)
    cols, vals = [], []
    for i in range(q.n):
        nz = np.nonzero(D[i])[0]
        cols.append(nz)
        vals.append(D[i, nz])
        rp[i + 1] = rp[i] + len(nz)
    lin = q.lin - b_pair / 2 * (np.arange(q.n) < 2 * (q.n // 2))
    return inputs.QuboArrays(q.n, rp, np.concatenate(cols).astype(np.int32),
                             np.concatenate(vals), lin)


@pytest.mark.parametrize("prec", [sb.SB_J_FP32, sb.SB_J_BF16])
def test_dsb_sign_bytes_keep_exact_with_huge_couplings(prec):
    """Sign bytes read as sgn / 2 and take the doubled weight 2 J, which would
    overflow for |J| >= 2^127. With J = 2e38 on every row every dSB form must
    still equal the FP32-position gather bit for bit (the library then gathers
    positions); with J = 1e36 (sqrt(sum J^2) < 2^125) the sign-byte forms run
    and agree too. c0 scales the coupling sum back to O(1)."""
    base = inputs.random_qubo(300, 6, seed=12)
    for b_pair, c0 in ((-8e38, 1e-38), (-4e36, 1e-36)):
        q = _with_huge_pairs(base, b_pair)
        x0, y0 = inputs.random_state(q.n, 128, 81, 0.9)
        for R, rw in ((128, 0), (128, 2), (48, 0)):
            outs = []
            for signs in (1, 0):
                ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, prec)
                sb.sb_set_option(ctx, sb.SB_OPT_ROWS_PER_WARP, rw)
                sb.sb_set_option(ctx, sb.SB_OPT_DSB_SIGNS, signs)
                sb.sb_set_state(ctx, x0[:, :R].copy(), y0[:, :R].copy())
                sb.sb_advance(ctx, "dsb", 1.0, c0, 0.5, 12,
                              _sched(np.float32(np.linspace(0, 1, 12))))
                outs.append(sb.sb_get_state(ctx))
                sb.sb_destroy(ctx)
            assert np.all(np.isfinite(outs[0][0])) and np.all(np.isfinite(outs[0][1]))
            assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
