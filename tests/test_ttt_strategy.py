"""The time-to-target arithmetic of the bench (section "Results", Table 1)
against the oracle's TTT formulas written out per checkpoint (oracle/ttt.py):
a round runs each of two configurations up to a checkpoint or not at all, and
is repeated until every event has succeeded with probability q."""
import itertools
import math

import numpy as np

import bench
from oracle import ttt as ottt


def _brute(t_list, P_list, q):
    """Every (k_1, k_2), k = -1 meaning the configuration is not run; rounds
    from ttt_at with a unit run time, the slowest event deciding."""
    (t1, t2), (P1, P2) = t_list, P_list
    best, arg = math.inf, None
    for k1, k2 in itertools.product(range(-1, len(t1)), range(-1, len(t2))):
        if k1 < 0 and k2 < 0:
            continue
        cost = (t1[k1] if k1 >= 0 else 0.0) + (t2[k2] if k2 >= 0 else 0.0)
        need = 0.0
        for e in range(P1.shape[1]):
            p = 1.0 - (1.0 - (P1[k1, e] if k1 >= 0 else 0.0)) * (1.0 - (P2[k2, e] if k2 >= 0 else 0.0))
            need = max(need, ottt.ttt_at(1.0, p, q))
        if cost * need < best:
            best, arg = cost * need, (k1, k2)
    return best, arg


def test_one_configuration_is_the_oracle_ttt():
    """The second configuration never succeeds: the best round is the oracle's
    min_k t(k) max(1, ln(1 - q) / ln(1 - p(k)))."""
    t1 = np.array([1.0, 2.0, 3.0, 4.0])
    p1 = np.array([0.0, 0.05, 0.4, 0.995])
    t2 = np.array([5.0, 10.0])
    got, ks = bench.ttt_strategy([t1, t2], [p1[:, None], np.zeros((2, 1))], 0.99)
    want = min(ottt.ttt_at(t, p, 0.99) for t, p in zip(t1, p1))
    assert math.isclose(got, want, rel_tol=1e-12) and ks[1] == -1
    # a batched run of R replicas succeeds with p_batch
    R = 64
    Pb = np.array([ottt.p_batch(p, R) for p in [0.0, 0.01, 0.02, 0.03]])
    got, _ = bench.ttt_strategy([t1, t2], [Pb[:, None], np.zeros((2, 1))], 0.99)
    assert math.isclose(got, min(ottt.ttt_at(t, p, 0.99) for t, p in zip(t1, Pb)), rel_tol=1e-12)


def test_events_reached_by_different_configurations_need_both():
    """Event 0 is reached only by configuration 1, event 1 only by
    configuration 2: no single configuration reaches both, a round of both
    does."""
    t1, t2 = np.array([1.0, 2.0]), np.array([3.0, 6.0])
    P1 = np.array([[0.0, 0.0], [0.5, 0.0]])
    P2 = np.array([[0.0, 0.2], [0.0, 0.9]])
    got, ks = bench.ttt_strategy([t1, t2], [P1, P2], 0.99)
    assert ks[0] >= 0 and ks[1] >= 0
    want, arg = _brute([t1, t2], [P1, P2], 0.99)
    assert math.isclose(got, want, rel_tol=1e-12) and ks == arg
    # no round reaches an event that neither configuration ever reaches
    P2[:, 1] = 0.0
    assert bench.ttt_strategy([t1, t2], [P1, P2], 0.99)[0] == math.inf


def test_random_cases_against_brute_force():
    rng = np.random.default_rng(7)
    for _ in range(30):
        n1, n2, E = rng.integers(1, 6), rng.integers(1, 6), rng.integers(1, 5)
        t1 = np.cumsum(rng.uniform(0.1, 1.0, n1))
        t2 = np.cumsum(rng.uniform(0.1, 1.0, n2))
        P1 = np.where(rng.uniform(size=(n1, E)) < 0.3, 0.0, rng.uniform(size=(n1, E)))
        P2 = np.where(rng.uniform(size=(n2, E)) < 0.3, 0.0, rng.uniform(size=(n2, E)))
        q = 0.99 ** (1.0 / E)
        got, ks = bench.ttt_strategy([t1, t2], [P1, P2], q)
        want, arg = _brute([t1, t2], [P1, P2], q)
        if want == math.inf:
            assert got == math.inf
        else:
            assert math.isclose(got, want, rel_tol=1e-12)
