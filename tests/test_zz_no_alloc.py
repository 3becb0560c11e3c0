"""sb_energy_noalloc -- the readout for callers that cannot allocate device
memory (host frameworks that own every device allocation under a fixed
budget, or latency-bound loops that cannot absorb cudaMalloc's implicit
synchronisation) -- against the allocating readout (sb_energy / sb_best),
through the C ABI, on two calls in a row that share the static scratch.

Kept in a file of its own, collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from paper_2402_14718_gb300.workloads import WORKLOADS
from oracle import events as oev, ising, qubo as oq

pytestmark = pytest.mark.gpu


def _qubo(name):
    w = WORKLOADS[name]
    ev = sb.sb_event_generate(w["seed"], sb.event_params(n_tracks=w["n_tracks"],
                                                         noise_frac=w["noise_frac"]))
    return sb.sb_qubo_build(ev, sb.build_params(**w["cuts"]))


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def test_noalloc_readout_matches_allocating_readout_twice():
    q = _qubo("event100")
    ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_FP32)
    d_rowptr, d_col = _dev(q.rowptr, torch.int32), _dev(q.col, torch.int32)
    d_qval, d_qlin = _dev(q.val, torch.float64), _dev(q.lin, torch.float64)
    # call 1: 64 replicas from positions x; call 2: 7 replicas from spins
    for R, seed, use_x in ((64, 3, True), (7, 4, False)):
        sb.sb_run(ctx, "bsb", 1.0, 0.0, 0.5, 150, R, seed=seed)
        x, _ = sb.sb_get_state(ctx)
        E_ref = sb.sb_energy(ctx, None, R)[0]
        _, bE_ref, br_ref = sb.sb_best(ctx)
        d_E = torch.full((R,), np.nan, dtype=torch.float64, device="cuda")
        d_bE = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        d_br = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        if use_x:
            d_x, d_s = _dev(x, torch.float32), None
        else:
            d_x, d_s = None, _dev(np.where(x > 0, 1, -1).astype(np.int8), torch.int8)
        sb.sb_energy_noalloc(q.n, d_rowptr, d_col, d_qval, d_qlin, d_x, d_s, R, d_E, d_bE, d_br)
        torch.cuda.synchronize()
        E = d_E.cpu().numpy()
        np.testing.assert_allclose(E, E_ref, rtol=1e-12, atol=1e-12)
        assert float(d_bE.item()) == pytest.approx(float(bE_ref[0]), rel=1e-12, abs=1e-12)
        assert int(d_br.item()) == int(br_ref[0])


def test_noalloc_readout_matches_the_oracle_energy():
    """Eq. 13 evaluated by its definition on the oracle's own QUBO of the same
    event, for seeded spins."""
    w = WORKLOADS["event100"]
    q = _qubo("event100")
    kw = dict(w["cuts"])
    kw["five_hit_rule"] = bool(kw["five_hit_rule"])
    qo = oq.build_qubo(oev.generate(w["seed"], oev.EventParams(n_tracks=w["n_tracks"],
                                                               noise_frac=w["noise_frac"])),
                       oq.BuildParams(**kw))
    R = 5
    T = np.random.default_rng(17).integers(0, 2, size=(qo.n, R)).astype(np.int8)
    d_E = torch.zeros(R, dtype=torch.float64, device="cuda")
    sb.sb_energy_noalloc(q.n, _dev(q.rowptr, torch.int32), _dev(q.col, torch.int32),
                         _dev(q.val, torch.float64), _dev(q.lin, torch.float64), None,
                         _dev(np.where(T > 0, 1, -1).astype(np.int8), torch.int8), R, d_E)
    torch.cuda.synchronize()
    np.testing.assert_allclose(d_E.cpu().numpy(), ising.qubo_energy(qo, T), rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    n, R = 300000, 256
    d_rowptr = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    d_qlin = torch.zeros(n, dtype=torch.float64, device="cuda")
    d_col = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_qval = torch.zeros(1, dtype=torch.float64, device="cuda")
    d_x = torch.zeros(1, dtype=torch.float32, device="cuda")
    d_E = torch.zeros(R, dtype=torch.float64, device="cuda")
    with pytest.raises(sb.SbError) as ei:
        sb.sb_energy_noalloc(n, d_rowptr, d_col, d_qval, d_qlin, d_x, None, R, d_E)
    assert ei.value.code == 1 and "static scratch" in str(ei.value)
    # a NULL column or value array is refused before any launch
    with pytest.raises(sb.SbError) as ei:
        sb.sb_energy_noalloc(100, d_rowptr, None, d_qval, d_qlin, d_x, None, 1, d_E)
    assert ei.value.code == 1
