"""Pins of the FP64 oracle adjoint of the bSB trajectory: central finite
differences of the oracle's own forward loss (h = 1e-6), at points where the
wall-mask sequence is the same on both sides of the difference."""
import numpy as np
import pytest

from oracle import adjoint, events, qubo, sb as osb
from paper_2402_14718_gb300.workloads import CUTS_S8


def _problem(n_tracks=40, seed=5):
    kw = dict(CUTS_S8)
    kw["five_hit_rule"] = True
    q = qubo.build_qubo(events.generate(seed, events.EventParams(n_tracks=n_tracks)),
                        qubo.BuildParams(**kw))
    return adjoint.Problem(q.n, q.rowptr, q.col, q.cls, q.quality)


def _fd(f, v, h=1e-6):
    return (f(v + h) - f(v - h)) / (2 * h)


@pytest.mark.parametrize("S", [12, 60])
def test_adjoint_matches_central_differences(S):
    p = _problem()
    R = 3
    x0, y0 = osb.init_state(7, p.n, R)
    sched = osb.linear_schedule(1.0, S)
    a0, c0, dt, wq, wc = 1.0, 0.3, 0.5, 1.0, 1.0
    loss, g = adjoint.gradient(p, x0, y0, sched, a0, c0, dt, wq, wc)
    assert loss == pytest.approx(adjoint.loss_only(p, x0, y0, sched, a0, c0, dt, wq, wc), rel=1e-14)
    h = 1e-6
    checks = {
        "dt": lambda v: adjoint.loss_only(p, x0, y0, sched, a0, c0, v, wq, wc),
        "c0": lambda v: adjoint.loss_only(p, x0, y0, sched, a0, v, dt, wq, wc),
        "w_q": lambda v: adjoint.loss_only(p, x0, y0, sched, a0, c0, dt, v, wc),
        "w_c": lambda v: adjoint.loss_only(p, x0, y0, sched, a0, c0, dt, wq, v),
    }
    base = {"dt": dt, "c0": c0, "w_q": wq, "w_c": wc}
    mkw = dict(a0=a0, c0=c0, dt=dt, w_q=wq, w_c=wc)
    checked = []
    for name, f in checks.items():
        lo, hi = dict(mkw), dict(mkw)
        lo[name] = base[name] - h
        hi[name] = base[name] + h
        same = np.array_equal(adjoint.masks(p, x0, y0, sched, **lo), adjoint.masks(p, x0, y0, sched, **hi))
        if not same:
            continue  # a wall event flips inside +-h: the loss has a kink there
        fd = _fd(f, base[name], h)
        assert g[name] == pytest.approx(fd, rel=1e-5, abs=1e-7), name
        checked.append(name)
    # a wall kink may excuse one scalar, not all of them
    assert len(checked) >= 3, checked
    rng = np.random.default_rng(S)
    for k in rng.choice(S, 5, replace=False):
        def fk(v, k=k):
            s2 = sched.copy()
            s2[k] = v
            return adjoint.loss_only(p, x0, y0, s2, a0, c0, dt, wq, wc)
        fd = _fd(fk, sched[k], h)
        assert g["sched"][k] == pytest.approx(fd, rel=1e-5, abs=1e-7)


def test_adjoint_loss_is_the_relaxed_energy():
    p = _problem(20, 3)
    J, h, _, _ = adjoint.weights(p, 1.0, 1.0)
    x, y = osb.init_state(1, p.n, 2)
    _, _, _, loss = adjoint.forward(J, h, x, y, [], 1.0, 0.5, 0.5)
    E = [float(-0.5 * x[:, r] @ (J @ x[:, r]) - h @ x[:, r]) for r in range(2)]
    assert loss == pytest.approx(np.mean(E), rel=1e-14)
    # the weights reproduce the builder's Ising field
    from oracle import ising
    kw = dict(CUTS_S8)
    kw["five_hit_rule"] = True
    q = qubo.build_qubo(events.generate(3, events.EventParams(n_tracks=20)), qubo.BuildParams(**kw))
    J2, h2, _ = ising.to_ising(q)
    np.testing.assert_allclose(h, h2, rtol=0, atol=1e-15)
    assert np.array_equal(J.data, J2.data)
