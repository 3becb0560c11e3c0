"""Host C++ generator, triplet-QUBO builder and track scorer against the FP64
oracle: integer and index arrays must be identical and every double equal
(bit-exact), on the same seeds and cuts."""
import numpy as np
import pytest

import paper_2402_14718_gb300 as sb
from paper_2402_14718_gb300.workloads import CUTS_PAPER, CUTS_S2_8, CUTS_S8
from oracle import events as oev
from oracle import qubo as oq
from oracle import tracks as otr


def _both_events(seed, n_tracks, noise):
    ev_c = sb.sb_event_generate(seed, sb.event_params(n_tracks=n_tracks, noise_frac=noise))
    ev_o = oev.generate(seed, oev.EventParams(n_tracks=n_tracks, noise_frac=noise))
    return ev_c, ev_o


@pytest.mark.parametrize("seed,n_tracks,noise", [(0, 100, 0.1), (7, 37, 0.0), (3000, 500, 0.1),
                                                 (4000, 60, 0.2)])
def test_event_generator_bit_exact(seed, n_tracks, noise):
    ev_c, ev_o = _both_events(seed, n_tracks, noise)
    a = ev_c.arrays()
    assert ev_c.n_true == ev_o.n_true
    np.testing.assert_array_equal(a["layer"], np.array(ev_o.layer, np.int32))
    np.testing.assert_array_equal(a["particle"], np.array(ev_o.particle, np.int32))
    for k in ("r", "phi", "z", "x", "y"):
        assert np.array_equal(a[k], np.array(getattr(ev_o, k))), k


def _cmp_qubo(qc, qo):
    assert qc.n == qo.n
    np.testing.assert_array_equal(qc.rowptr, qo.rowptr)
    np.testing.assert_array_equal(qc.col, qo.col)
    assert np.array_equal(qc.val, qo.val)
    assert np.array_equal(qc.lin, qo.lin)
    assert np.array_equal(qc.quality, qo.quality)
    assert np.array_equal(qc.kappa, qo.kappa)
    assert np.array_equal(qc.dtheta, qo.dtheta)
    np.testing.assert_array_equal(qc.cls, qo.cls)
    np.testing.assert_array_equal(qc.trip, qo.trip)


@pytest.mark.parametrize("seed,n_tracks,noise,cuts", [(0, 100, 0.1, CUTS_S8),
                                                      (0, 100, 0.1, CUTS_PAPER),
                                                      (3000, 500, 0.1, CUTS_S2_8)])
def test_qubo_builder_bit_exact(seed, n_tracks, noise, cuts):
    ev_c, ev_o = _both_events(seed, n_tracks, noise)
    qc = sb.sb_qubo_build(ev_c, sb.build_params(**cuts))
    kw = dict(cuts)
    kw["five_hit_rule"] = bool(kw["five_hit_rule"])
    qo = oq.build_qubo(ev_o, oq.BuildParams(**kw))
    assert qc.n > 0
    _cmp_qubo(qc, qo)


def test_builder_without_five_hit_rule_and_weights():
    ev_c, ev_o = _both_events(5, 80, 0.1)
    kw = dict(CUTS_S8, w_q=0.7, w_c=2.5, five_hit_rule=0)
    qc = sb.sb_qubo_build(ev_c, sb.build_params(**kw))
    kw["five_hit_rule"] = False
    qo = oq.build_qubo(ev_o, oq.BuildParams(**kw))
    _cmp_qubo(qc, qo)
    assert set(np.unique(qc.val)) <= {-1.0, 2.5}


@pytest.mark.parametrize("frac", [0.0, 0.3, 0.7, 1.0])
def test_tracks_and_scores_bit_exact(frac):
    ev_c, ev_o = _both_events(0, 100, 0.1)
    qc = sb.sb_qubo_build(ev_c, sb.build_params(**CUTS_S8))
    kw = dict(CUTS_S8)
    kw["five_hit_rule"] = True
    qo = oq.build_qubo(ev_o, oq.BuildParams(**kw))
    rng = np.random.default_rng(int(frac * 10))
    T = (rng.random(qc.n) < frac).astype(np.uint8)
    truth = np.array([1 if ev_o.particle[a] == ev_o.particle[b] == ev_o.particle[c] >= 0 else 0
                      for (a, b, c) in qo.trip], np.uint8)
    for sel in (T, truth, T | truth):
        rc = sb.sb_tracks(ev_c, qc, sel)
        tr, reco = otr.assemble(qo, sel)
        tp, fp, fn, eff, pur = otr.score(ev_o, reco)
        assert rc["tracks"] == tr
        assert (rc["tp"], rc["fp"], rc["fn"]) == (tp, fp, fn)
        assert rc["efficiency"] == eff and rc["purity"] == pur


@pytest.mark.parametrize("cm,bm", [(1, 0), (0, 1), (1, 1)])
def test_paper_weights_bit_exact(cm, bm):
    ev_c, ev_o = _both_events(0, 100, 0.1)
    kw = dict(CUTS_S8, coupling_mode=cm, bias_mode=bm)
    qc = sb.sb_qubo_build(ev_c, sb.build_params(**kw))
    kw["five_hit_rule"] = True
    qo = oq.build_qubo(ev_o, oq.BuildParams(**kw))
    _cmp_qubo(qc, qo)
    if cm:
        cons = qc.val[qc.cls == 0]
        assert np.all((cons < -0.2) & (cons >= -1.0)) and len(np.unique(cons)) > 10
