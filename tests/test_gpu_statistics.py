"""Statistics over independent starts in the bench's configurations: the
500-track event with BF16 J and the factored coupling product (R = 128: the
row-group kernel over the extended CSR for bSB, the factored sign-byte kernel
for dSB), against the FP64 oracle over the same 128 starts and the same
schedule: median final QUBO energy within 0.5 %, efficiency and purity of
the best replica within one point (trajectories themselves diverge with FP32
rounding, so only these statistics are compared)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from oracle import ising, sb as osb, tracks as otr
from tests.gpu_common import oracle_c0, workload_qubos

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [osb.BSB, osb.DSB])
def test_statistics_event500_bf16_factored(variant):
    ev_c, qc, ev_o, qo = workload_qubos("event500")
    R, S = 128, 1000
    name = {osb.BSB: "bsb", osb.DSB: "dsb"}[variant]
    ctx = sb.sb_create(qc.n, qc.rowptr, qc.col, qc.val, qc.lin, sb.SB_J_BF16)
    member, couple, w, n_ids = sb.sb_qubo_factor(qc)
    sb.sb_set_factor(ctx, n_ids, member, couple, w)
    c0 = oracle_c0(qo)
    sb.sb_run(ctx, name, 1.0, c0, 0.5, S, R, seed=515)
    E_gpu = sb.sb_energy(ctx, None, R)[0]
    T_g, _, _ = sb.sb_best(ctx)
    J, h, _ = ising.to_ising(qo)
    x, y = osb.init_state(515, qo.n, R)
    res = osb.run(J, h, x, y, osb.linear_schedule(1.0, S), 1.0, c0, 0.5, variant)
    T_o = ising.triplets_from_spins(ising.spins_from_x(res.x))
    E_orc = ising.qubo_energy(qo, T_o)
    med_g, med_o = float(np.median(E_gpu)), float(np.median(E_orc))
    assert abs(med_g - med_o) <= 0.005 * abs(med_o), (med_g, med_o)
    sc_g = sb.sb_tracks(ev_c, qc, T_g)
    _, reco = otr.assemble(qo, T_o[:, int(np.argmin(E_orc))])
    _, _, _, eff_o, pur_o = otr.score(ev_o, reco)
    assert abs(sc_g["efficiency"] - eff_o) <= 0.01
    assert abs(sc_g["purity"] - pur_o) <= 0.01
