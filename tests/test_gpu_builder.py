"""The triplet-QUBO builder on the GPU against the host builder (which is
bit-exact with the FP64 oracle): identical triplets, rows, columns and classes;
values identical up to the last place where they pass through atan2 or exp."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2402_14718_gb300 as sb
from paper_2402_14718_gb300.workloads import CUTS_DENSE, CUTS_PAPER, CUTS_S2_35, CUTS_S2_8, CUTS_S8

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,tracks,noise,cuts,extra", [
    (0, 100, 0.1, CUTS_S8, {}),
    (0, 100, 0.1, CUTS_PAPER, {}),
    (0, 100, 0.1, CUTS_S8, dict(coupling_mode=1, bias_mode=1)),
    (7, 37, 0.0, CUTS_S8, dict(five_hit_rule=0, w_c=2.5, w_q=0.7)),
    (1000, 1000, 0.1, CUTS_S2_35, {}),
    (4000, 3000, 0.2, CUTS_DENSE, {}),
])
def test_device_builder_matches_host(seed, tracks, noise, cuts, extra):
    ev = sb.sb_event_generate(seed, sb.event_params(n_tracks=tracks, noise_frac=noise))
    p = sb.build_params(**dict(cuts, **extra))
    qh = sb.sb_qubo_build(ev, p)
    qd, ms = sb.sb_qubo_build_device(ev, p)
    assert ms > 0
    assert qd.n == qh.n and qd.nnz == qh.nnz
    for k in ("rowptr", "col", "cls", "trip"):
        np.testing.assert_array_equal(getattr(qd, k), getattr(qh, k), err_msg=k)
    assert np.array_equal(qd.kappa, qh.kappa)       # +, -, *, /, sqrt only: bit-exact
    for k in ("val", "lin", "quality", "dtheta"):
        np.testing.assert_allclose(getattr(qd, k), getattr(qh, k), rtol=1e-12, atol=1e-15,
                                   err_msg=k)


def test_device_builder_empty_and_tiny_events():
    ev = sb.sb_event_generate(1, sb.event_params(n_tracks=0))
    q, _ = sb.sb_qubo_build_device(ev, sb.build_params(**CUTS_S8))
    assert q.n == 0 and q.nnz == 0
    ev = sb.sb_event_generate(2, sb.event_params(n_tracks=1, noise_frac=0.0))
    qd, _ = sb.sb_qubo_build_device(ev, sb.build_params(**CUTS_S8))
    qh = sb.sb_qubo_build(ev, sb.build_params(**CUTS_S8))
    assert qd.n == qh.n == 8 and np.array_equal(qd.col, qh.col)


@pytest.mark.parametrize("seed,tracks,noise,cuts,extra", [
    (0, 100, 0.1, CUTS_S8, {}),
    (0, 100, 0.1, CUTS_S8, dict(coupling_mode=1, bias_mode=1)),
    (7, 37, 0.0, CUTS_S8, dict(five_hit_rule=0, w_c=2.5, w_q=0.7)),
    (3000, 500, 0.1, CUTS_S2_8, {}),
])
def test_device_builder_matches_oracle(seed, tracks, noise, cuts, extra):
    """The GPU builder against the FP64 oracle's builder directly: the same
    triplets, rows, columns and classes; values to 1e-12 (the FP64 atan2 / exp
    of the device may differ from the host's libm in the last place)."""
    from oracle import events as oev, qubo as oq
    ev = sb.sb_event_generate(seed, sb.event_params(n_tracks=tracks, noise_frac=noise))
    qd, _ = sb.sb_qubo_build_device(ev, sb.build_params(**dict(cuts, **extra)))
    kw = dict(cuts, **extra)
    kw["five_hit_rule"] = bool(kw["five_hit_rule"])
    qo = oq.build_qubo(oev.generate(seed, oev.EventParams(n_tracks=tracks, noise_frac=noise)),
                       oq.BuildParams(**kw))
    assert qd.n == qo.n
    for k in ("rowptr", "col", "cls", "trip"):
        np.testing.assert_array_equal(getattr(qd, k), getattr(qo, k), err_msg=k)
    np.testing.assert_allclose(qd.kappa, qo.kappa, rtol=1e-12, atol=0)
    for k in ("val", "lin", "quality", "dtheta"):
        np.testing.assert_allclose(getattr(qd, k), getattr(qo, k), rtol=1e-12, atol=1e-15,
                                   err_msg=k)
