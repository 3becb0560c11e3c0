"""bSB adjoint on the GPU (sb_backward through the C ABI) against the FP64
oracle adjoint, which itself is pinned by central finite differences.

Long bSB runs are chaotic (FP32 and FP64 trajectories part after a few hundred
steps), so GPU and oracle gradients are compared on short horizons, at the
problem sizes of the workloads; tolerance 1e-3 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from oracle import adjoint, sb as osb
from tests.gpu_common import workload_qubos

pytestmark = pytest.mark.gpu


def _oracle(qo, R, S, seed, c0, dt, w_q=1.0, w_c=1.0, sched=None):
    p = adjoint.Problem(qo.n, qo.rowptr, qo.col, qo.cls, qo.quality)
    x0, y0 = osb.init_state(seed, qo.n, R)
    if sched is None:
        sched = np.float32(osb.linear_schedule(1.0, S)).astype(np.float64)
    return adjoint.gradient(p, x0, y0, sched, 1.0, c0, dt, w_q, w_c)


def _gpu(qc, R, S, seed, c0, dt, K, prec=sb.SB_J_FP32, w_q=1.0, w_c=1.0, sched=None):
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, prec)
    sb.sb_set_weights(ctx, qc.cls, qc.quality, w_q, w_c)
    if sched is None:
        sched = np.float32(osb.linear_schedule(1.0, S))
    d_sched = torch.tensor(np.asarray(sched, np.float32), device="cuda")
    g_a = torch.zeros(S, dtype=torch.float64, device="cuda")
    loss, g = sb.sb_backward(ctx, 1.0, c0, dt, S, R, seed, d_sched, K, g_a)
    g["sched"] = g_a.cpu().numpy()
    return loss, g


def _close(gg, go, rel=1e-3):
    for k in ("dt", "c0", "w_q", "w_c"):
        assert gg[k] == pytest.approx(go[k], rel=rel, abs=rel * 1e-3), k
    scale = np.max(np.abs(go["sched"]))
    assert np.max(np.abs(gg["sched"] - go["sched"])) <= rel * scale


@pytest.mark.parametrize("S,K", [(30, 8), (30, 30), (45, 1), (30, 64)])
def test_adjoint_matches_oracle_event100(S, K):
    _, qc, _, qo = workload_qubos("event100")
    lg, gg = _gpu(qc, 8, S, 3, 0.3, 0.5, K)
    lo, go = _oracle(qo, 8, S, 3, 0.3, 0.5)
    assert lg == pytest.approx(lo, rel=1e-4)
    _close(gg, go)


def test_adjoint_weight_scales_and_bf16():
    _, qc, _, qo = workload_qubos("event100")
    lg, gg = _gpu(qc, 4, 25, 9, 0.25, 0.5, 6, prec=sb.SB_J_BF16, w_q=0.7, w_c=2.0)
    lo, go = _oracle(qo, 4, 25, 9, 0.25, 0.5, w_q=0.7, w_c=2.0)
    assert lg == pytest.approx(lo, rel=1e-4)
    _close(gg, go)


def test_adjoint_full_event500_shape_short_horizon():
    """The 500-track workload (N ~ 10.9k, R = 32, checkpoint every 32 steps) on
    a 40-step horizon."""
    _, qc, _, qo = workload_qubos("event500")
    lg, gg = _gpu(qc, 32, 40, 11, 0.3, 0.5, 32)
    lo, go = _oracle(qo, 32, 40, 11, 0.3, 0.5)
    assert lg == pytest.approx(lo, rel=1e-4)
    _close(gg, go)


def test_checkpoint_interval_does_not_change_gradients():
    _, qc, _, _ = workload_qubos("event500")
    ref = None
    for K in (1, 32, 100, 250):
        loss, g = _gpu(qc, 32, 250, 2, 0.3, 0.5, K)
        if ref is None:
            ref = (loss, g)
            continue
        # FP64 block sums are combined with atomics: order-dependent in the last place
        assert loss == pytest.approx(ref[0], rel=1e-13)
        for k in ("dt", "c0", "w_q", "w_c"):
            assert g[k] == pytest.approx(ref[1][k], rel=1e-9, abs=1e-12)
        np.testing.assert_allclose(g["sched"], ref[1]["sched"], rtol=1e-9, atol=1e-12)


def test_autograd_function_full_workload():
    """torch.autograd.Function over the full 500-track workload: 1000 steps,
    32 replicas, checkpoint every 32; gradients flow to every input."""
    _, qc, _, _ = workload_qubos("event500")
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_FP32)
    S = 1000
    dt = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    c0 = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    a = torch.tensor(np.float32(osb.linear_schedule(1.0, S)), requires_grad=True)
    wq = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    wc = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    loss = sb.SBRelaxedEnergy.apply(dt, c0, a, wq, wc, ctx, qc.cls, qc.quality, 32, 5, 32)
    loss.backward()
    l2, g2 = sb.sb_backward(ctx, 1.0, 0.3, 0.5, S, 32, 5, a.detach().cuda(), 32)
    # the loss is an FP64 sum combined with atomics between blocks: last-bit order effects
    assert float(loss.detach()) == pytest.approx(l2, rel=1e-13)
    assert float(dt.grad) == pytest.approx(g2["dt"], rel=1e-9)
    assert float(wc.grad) == pytest.approx(g2["w_c"], rel=1e-9)
    assert a.grad.shape == (S,) and torch.isfinite(a.grad).all()
    assert all(torch.isfinite(t.grad) for t in (dt, c0, wq, wc))


def test_work_memory_kept_between_calls_of_one_shape():
    """sb_backward keeps its work memory for the next call of the same shape
    and reallocates on another shape; results repeat (to the FP64 atomics'
    ordering) whichever call comes first."""
    _, qc, _, qo = workload_qubos("event100")
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_FP32)
    sb.sb_set_weights(ctx, qc.cls, qc.quality, 1.0, 1.0)

    def run(S, R, K):
        d_sched = torch.tensor(np.float32(osb.linear_schedule(1.0, S)), device="cuda")
        g_a = torch.zeros(S, dtype=torch.float64, device="cuda")
        loss, g = sb.sb_backward(ctx, 1.0, 0.3, 0.5, S, R, 3, d_sched, K, g_a)
        g["sched"] = g_a.cpu().numpy()
        return loss, g

    first = run(30, 8, 8)
    for shape in ((30, 8, 8), (30, 8, 5), (31, 8, 8), (30, 16, 8), (30, 8, 8)):
        again = run(*shape)
        if shape == (30, 8, 8):
            assert again[0] == pytest.approx(first[0], rel=1e-13)
            _close(again[1], first[1], rel=1e-10)
    lo, go = _oracle(qo, 8, 30, 3, 0.3, 0.5)
    assert first[0] == pytest.approx(lo, rel=1e-4)
    _close(first[1], go)


def test_one_replica_lane_groups_in_the_adjoint():
    """The recording step of sb_backward at R = 1 with lane groups gives the
    gradients of the one-thread form (to the FP64 atomics' ordering)."""
    _, qc, _, qo = workload_qubos("event100")
    out = []
    for lanes in (16, 0):
        ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_FP32)
        sb.sb_set_weights(ctx, qc.cls, qc.quality, 1.0, 1.0)
        sb.sb_set_option(ctx, sb.SB_OPT_R1_LANES, lanes)
        d_sched = torch.tensor(np.float32(osb.linear_schedule(1.0, 30)), device="cuda")
        g_a = torch.zeros(30, dtype=torch.float64, device="cuda")
        loss, g = sb.sb_backward(ctx, 1.0, 0.3, 0.5, 30, 1, 3, d_sched, 8, g_a)
        g["sched"] = g_a.cpu().numpy()
        out.append((loss, g))
        sb.sb_destroy(ctx)
    assert out[0][0] == pytest.approx(out[1][0], rel=1e-13)
    _close(out[0][1], out[1][1], rel=1e-10)
    lo, go = _oracle(qo, 1, 30, 3, 0.3, 0.5)
    assert out[0][0] == pytest.approx(lo, rel=1e-4)
    _close(out[0][1], go)
