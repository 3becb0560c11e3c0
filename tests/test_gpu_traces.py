"""Energy traces (the Fig. 2 / Fig. 4 analogue of the paper-size study): the
FP64 QUBO energies the library reports at trace checkpoints equal Eq. 13 by
definition (the oracle, on its own QUBO of the same event) for the spins read
back at those checkpoints."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from paper_2402_14718_gb300.workloads import CUTS_DENSE, PAPER_SIZES
from oracle import events as oev, ising, qubo as oq

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["bsb", "dsb"])
def test_trace_checkpoint_energies_match_oracle(variant):
    p = PAPER_SIZES[0]
    ev = sb.sb_event_generate(p["seed"], sb.event_params(n_tracks=p["n_tracks"]))
    q = sb.sb_qubo_build(ev, sb.build_params(**CUTS_DENSE))
    kw = dict(CUTS_DENSE)
    kw["five_hit_rule"] = bool(kw["five_hit_rule"])
    qo = oq.build_qubo(oev.generate(p["seed"], oev.EventParams(n_tracks=p["n_tracks"])),
                       oq.BuildParams(**kw))
    assert q.n == qo.n == 779 and np.array_equal(q.col, qo.col)
    R, S, every = 16, 300, 100
    ctx = sb.sb_create(q.n, q.rowptr, q.col, q.val, q.lin, sb.SB_J_BF16)
    sched = torch.tensor(np.array([k / (S - 1) for k in range(S)], np.float32), device="cuda")
    sb.sb_run(ctx, variant, 1.0, 0.0, 1.0, 0, R, seed=1)
    for k0 in range(0, S, every):
        sb.sb_advance(ctx, variant, 1.0, 0.0, 1.0, every, sched[k0:k0 + every])
        E_gpu = sb.sb_energy(ctx, None, R)[0]
        x, _ = sb.sb_get_state(ctx)
        E_orc = ising.qubo_energy(qo, ising.triplets_from_spins(ising.spins_from_x(x)))
        np.testing.assert_allclose(E_gpu, E_orc, rtol=1e-12, atol=1e-12)
