"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published known-answer vectors, Lorentz-force geometry, exhaustive search,
Hamiltonian conservation of Eq. 3-4 / 7-8, closed forms and special cases."""
import math
import os

import numpy as np
import pytest

from oracle import philox, events, qubo, ising, sb, bruteforce, tracks, ttt
from tests.inputs import random_qubo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Known-answer vectors published with the Random123 library (Philox4x32-10)."""
    path = os.path.join(GOLDEN, "philox4x32_10_kat.txt")
    n = 0
    for line in open(path):
        line = line.split("#")[0].split()
        if not line:
            continue
        ins = [int(v, 16) for v in line[:6]]
        expect = [int(v, 16) for v in line[6:10]]
        assert list(philox.philox4x32_10(*ins)) == expect
        n += 1
    assert n == 3


def test_uniform_range_and_resolution():
    assert philox.uniform01(0, 0) == 0.0
    assert philox.uniform01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert philox.uniform01(1 << 11, 0) == 2.0 ** -53


# ---------------------------------------------------------------- events
def _clean_params(n):
    return events.EventParams(n_tracks=n, noise_frac=0.0, smear_rphi=0.0, smear_z=0.0)


def test_hits_lie_on_lorentz_circle_and_helix():
    """A charge q in B = +z turns clockwise for q > 0: the transverse circle has
    centre q Rc (sin phi0, -cos phi0) and passes through the origin; z grows
    linearly with the transverse arc length, dz/ds = sinh(eta)."""
    ev = events.generate(7, _clean_params(20))
    hits_by_track = {}
    for h, part in enumerate(ev.particle):
        hits_by_track.setdefault(part, []).append(h)
    for t, (q, pt, eta, phi0, z0, rc) in enumerate(ev.truth):
        assert rc == pytest.approx(pt / (0.3 * 2.0) * 1000.0, rel=1e-14)
        cx, cy = q * rc * math.sin(phi0), -q * rc * math.cos(phi0)
        for h in hits_by_track[t]:
            d = math.sqrt((ev.x[h] - cx) ** 2 + (ev.y[h] - cy) ** 2)
            assert d == pytest.approx(rc, rel=1e-9)
            assert math.sqrt(ev.x[h] ** 2 + ev.y[h] ** 2) == pytest.approx(ev.r[h], rel=1e-12)
            # arc length from the origin = Rc * (angle between centre->origin and centre->hit)
            v0 = (-cx, -cy)
            v1 = (ev.x[h] - cx, ev.y[h] - cy)
            ang = abs(math.atan2(v0[0] * v1[1] - v0[1] * v1[0], v0[0] * v1[0] + v0[1] * v1[1]))
            assert ev.z[h] - z0 == pytest.approx(rc * ang * math.sinh(eta), rel=1e-9, abs=1e-9)


def test_event_sorted_and_noise_count():
    ev = events.generate(3, events.EventParams(n_tracks=50, noise_frac=0.1))
    assert ev.n_true == 500
    assert len(ev.layer) == 550
    keys = list(zip(ev.layer, ev.phi))
    assert keys == sorted(keys)
    assert all(-math.pi <= p < math.pi for p in ev.phi)
    assert sum(1 for p in ev.particle if p < 0) == 50


# ---------------------------------------------------------------- builder
def test_curvature_of_points_on_a_known_circle():
    R = 1234.5
    pts = [(R * math.cos(a), R * math.sin(a) + 17.0) for a in (0.1, 0.35, 0.8)]
    k = qubo.curvature(*pts[0], *pts[1], *pts[2])
    assert k == pytest.approx(1.0 / R, rel=1e-12)          # counter-clockwise: +
    k2 = qubo.curvature(*pts[2], *pts[1], *pts[0])
    assert k2 == pytest.approx(-1.0 / R, rel=1e-12)
    assert qubo.curvature(0.0, 0.0, 1.0, 1.0, 2.0, 2.0) == 0.0


def _separated_seed(n_tracks, min_dphi):
    for seed in range(1000):
        ev = events.generate(seed, _clean_params(n_tracks))
        ph = sorted(t[3] for t in ev.truth)
        gaps = [ph[k + 1] - ph[k] for k in range(len(ph) - 1)] + [ph[0] + 2 * math.pi - ph[-1]]
        if min(gaps) > min_dphi:
            return seed, ev
    raise AssertionError("no separated event found")


def test_builder_on_isolated_clean_tracks():
    """Isolated, unsmeared tracks: every track gives its 8 triplets, each linked to
    its neighbours by 7 consistent pairs (b = -1), no conflict, and the triplet
    curvature is -q / Rc."""
    seed, ev = _separated_seed(4, 0.6)
    p = qubo.BuildParams(dphi_slope=1.5e-3, dphi_margin=1.0, z0_max=100, kappa_max=2e-3,
                         dtheta_max=0.2, dkappa_max=5e-4)
    q = qubo.build_qubo(ev, p)
    assert q.n == 8 * 4
    assert len(q.col) == 14 * 4
    assert np.all(q.val == -1.0)
    for i in range(q.n):
        a, b, c = q.trip[i]
        part = ev.particle[a]
        assert part == ev.particle[b] == ev.particle[c] >= 0
        qq, pt, eta, phi0, z0, rc = ev.truth[part]
        assert q.kappa[i] == pytest.approx(-qq / rc, rel=1e-6)
        # closed form from the truth helix: z - z0 = sinh(eta) * 2 Rc asin(r / 2Rc)
        def zs(h):
            return math.sinh(eta) * 2 * rc * math.asin(ev.r[h] / (2 * rc))
        th1 = math.atan2(ev.r[b] - ev.r[a], zs(b) - zs(a))
        th2 = math.atan2(ev.r[c] - ev.r[b], zs(c) - zs(b))
        assert q.dtheta[i] == pytest.approx(abs(th2 - th1), rel=1e-6, abs=1e-12)
    # CSR layout: ascending columns, symmetric, no diagonal
    for i in range(q.n):
        cols = q.col[q.rowptr[i]:q.rowptr[i + 1]]
        assert list(cols) == sorted(cols) and i not in cols


def test_conflict_rule_on_a_fork():
    """Two tracks crossing at a shared hit make forks: the pairs that share a hit
    on the same or adjacent start layers (and are not consistent) get +w_c."""
    ev = events.Event(layer=[], r=[], phi=[], z=[], x=[], y=[], particle=[], n_true=0)
    # five layers, two straight radial tracks at phi = 0 and phi = 0.001 sharing layer-2 hit
    radii = events.LAYER_RADII[:5]
    hits = []
    for l, r in enumerate(radii):
        hits.append((l, 0.0, 0.5 * r, 0))
        if l != 2:
            hits.append((l, 0.001, 0.5 * r, 1))
    hits.sort(key=lambda h: (h[0], h[1]))
    for (l, phi, z, part) in hits:
        r = radii[l]
        ev.layer.append(l); ev.r.append(r); ev.phi.append(phi); ev.z.append(z)
        ev.x.append(r * math.cos(phi)); ev.y.append(r * math.sin(phi)); ev.particle.append(part)
    p = qubo.BuildParams(dphi_slope=1e-3, dphi_margin=1.0, z0_max=100, kappa_max=2e-3,
                         dtheta_max=0.2, dkappa_max=5e-4, w_c=2.5, five_hit_rule=False)
    q = qubo.build_qubo(ev, p)
    B = bruteforce.dense_lower(q)
    B = B + B.T
    trip = [tuple(int(v) for v in t) for t in q.trip]
    for i, t in enumerate(trip):
        for j, u in enumerate(trip):
            if i == j:
                continue
            shared = set(t) & set(u)
            li, lj = ev.layer[t[0]], ev.layer[u[0]]
            if not shared or abs(li - lj) >= 2:
                assert B[i, j] == 0.0
            elif (lj == li + 1 and t[1:] == u[:2]) or (li == lj + 1 and u[1:] == t[:2]):
                assert B[i, j] == -1.0
            else:
                assert B[i, j] == 2.5


# ---------------------------------------------------------------- Ising map
def test_qubo_ising_identity_exhaustive():
    """O(T) (Eq. 13 by definition) == offset + E_ising(s) for every T, N = 12."""
    q = random_qubo(12, 4, seed=5, values=(-1.0, 1.0, 0.37))
    J, h, off = ising.to_ising(q)
    ids = np.arange(1 << q.n)
    T = ((ids[None, :] >> np.arange(q.n)[:, None]) & 1).astype(np.float64)
    E_q = ising.qubo_energy(q, T)
    E_i = ising.ising_energy(J, h, 2.0 * T - 1.0) + off
    np.testing.assert_allclose(E_q, E_i, rtol=0, atol=1e-12)


def test_qubo_ising_identity_on_event():
    ev = events.generate(0, events.EventParams(n_tracks=100))
    q = qubo.build_qubo(ev, qubo.BuildParams(**_PRESET_100))
    J, h, off = ising.to_ising(q)
    rng = np.random.default_rng(1)
    T = rng.integers(0, 2, size=(q.n, 8)).astype(np.float64)
    E_q = ising.qubo_energy(q, T)
    E_i = ising.ising_energy(J, h, 2.0 * T - 1.0) + off
    np.testing.assert_allclose(E_q, E_i, rtol=1e-13, atol=1e-10)


def test_golden_five_hit_track():
    """Hand-computed Eq. 13 energies of a 3-triplet chain (tests/golden)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "chain3_energies.txt")) if l.strip() and not l.startswith("#")]
    # a = (0.2, 0.1, 0.3); b_01 = b_12 = -1, b_02 = 0 (junction hit only)
    from tests.inputs import QuboArrays
    q = QuboArrays(3, np.array([0, 1, 3, 4], np.int32), np.array([1, 0, 2, 1], np.int32),
                   np.array([-1.0, -1.0, -1.0, -1.0]), np.array([0.2, 0.1, 0.3]))
    for r in rows:
        T = np.array([int(c) for c in r[0]])
        assert ising.qubo_energy(q, T) == pytest.approx(float(r[1]), abs=1e-15)
    E, arg = bruteforce.ground_state(q)
    assert E == pytest.approx(-1.4) and [list(a) for a in arg] == [[1, 1, 1]]


# ---------------------------------------------------------------- brute force
def test_bruteforce_closed_forms():
    # no couplings: T_i = [a_i < 0]
    from tests.inputs import QuboArrays
    lin = np.array([0.5, -0.25, -1.0, 0.0, 2.0, -0.125])
    q = QuboArrays(6, np.zeros(7, np.int32), np.zeros(0, np.int32), np.zeros(0), lin)
    E, arg = bruteforce.ground_state(q)
    assert E == -1.375
    assert len(arg) == 2          # a_3 = 0: both choices are optimal
    # ferromagnetic chain with small positive bias: everything on
    n = 10
    rp = [0]; col = []
    for i in range(n):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        col += nb; rp.append(len(col))
    q = QuboArrays(n, np.array(rp, np.int32), np.array(col, np.int32), -np.ones(len(col)), np.full(n, 0.3))
    E, arg = bruteforce.ground_state(q)
    assert E == pytest.approx(0.3 * n - (n - 1))
    assert len(arg) == 1 and arg[0].sum() == n


def test_bruteforce_matches_plain_enumeration():
    import itertools
    q = random_qubo(9, 3, seed=11, values=(-1.0, 1.0, 0.5))
    best = math.inf
    for bits in itertools.product((0, 1), repeat=q.n):
        e = sum(q.lin[i] * bits[i] for i in range(q.n))
        for i in range(q.n):
            for p in range(q.rowptr[i], q.rowptr[i + 1]):
                if q.col[p] < i:
                    e += q.val[p] * bits[i] * bits[q.col[p]]
        best = min(best, e)
    E, _ = bruteforce.ground_state(q)
    assert E == pytest.approx(best, abs=1e-12)


# ---------------------------------------------------------------- SB dynamics
_PRESET_100 = dict(dphi_slope=3.2e-3, dphi_margin=4.0, z0_max=400, kappa_max=6.4e-3,
                   dtheta_max=0.8, dkappa_max=5e-4)


def _event_sub_qubo(q, start, n):
    """Rows start..start+n-1 of an event QUBO with the couplings inside the block."""
    from tests.inputs import QuboArrays
    rp, col, val = [0], [], []
    for i in range(start, start + n):
        for p in range(q.rowptr[i], q.rowptr[i + 1]):
            j = q.col[p]
            if start <= j < start + n:
                col.append(j - start)
                val.append(q.val[p])
        rp.append(len(col))
    return QuboArrays(n, np.array(rp, np.int32), np.array(col, np.int32), np.array(val),
                      q.lin[start:start + n].copy())


@pytest.fixture(scope="module")
def small_instances():
    ev = events.generate(0, events.EventParams(n_tracks=100))
    qe = qubo.build_qubo(ev, qubo.BuildParams(**_PRESET_100))
    out = []
    for inst in range(20):
        n = 12 + inst % 9
        out.append(("event", _event_sub_qubo(qe, 37 * inst % (qe.n - n), n)))
        out.append(("random", random_qubo(n, 3, seed=100 + inst, values=(-1.0, 1.0),
                                          lin_low=-0.5, lin_high=0.5)))
    return out


def _sb_ground_hits(instances, variant, R=64, S=2000):
    hits = {"event": 0, "random": 0}
    for k, (kind, q) in enumerate(instances):
        E0, _ = bruteforce.ground_state(q)
        J, h, off = ising.to_ising(q)
        c0 = ising.c0_auto(J, q.n)
        x, y = sb.init_state(k // 2, q.n, R)
        res = sb.run(J, h, x, y, sb.linear_schedule(1.0, S), 1.0, c0, 0.5, variant)
        T = ising.triplets_from_spins(ising.spins_from_x(res.x))
        E = ising.qubo_energy(q, T)
        hits[kind] += int(np.min(E) <= E0 + 1e-9)
    return hits


def test_bsb_reaches_exact_ground_state(small_instances):
    """64 replicas x 2000 steps: on tracking sub-QUBOs (N = 12..20) at least 95 %
    of the instances have a replica at the exhaustive ground energy; random
    frustrated +-1 QUBOs are harder for bSB (about 90 % measured)."""
    hits = _sb_ground_hits(small_instances, sb.BSB)
    assert hits["event"] >= 19
    assert hits["random"] >= 17


def test_dsb_reaches_exact_ground_state(small_instances):
    hits = _sb_ground_hits(small_instances, sb.DSB)
    assert hits["event"] >= 19
    assert hits["random"] >= 18


def test_wall_invariant_every_step():
    q = random_qubo(40, 5, seed=3)
    J, h, _ = ising.to_ising(q)
    x, y = sb.init_state(9, 40, 16)
    for variant in (sb.BSB, sb.DSB):
        xx, yy = x.copy(), y.copy()
        for a_k in sb.linear_schedule(1.0, 300):
            xx, yy = sb.step(J, h, xx, yy, a_k, 1.0, 2.0, 0.5, variant)
            assert np.max(np.abs(xx)) <= 1.0
            assert np.all(yy[np.abs(xx) == 1.0] == 0.0)
        assert np.any(np.abs(xx) == 1.0)


def test_free_particle_closed_forms():
    """J = 0, h = 0: with a = a0 the force vanishes, so y is constant and x moves
    linearly until the wall; with a = 0 the step is the linear map
    [[1 - (dt a0)^2, dt a0], [-dt a0, 1]] applied k times (matrix power)."""
    import scipy.sparse as sp
    n, R, dt, a0 = 5, 3, 0.05, 1.0
    J = sp.csr_matrix((n, n))
    h = np.zeros(n)
    x0, y0 = sb.init_state(1, n, R)
    x, y = x0.copy(), y0.copy()
    for k in range(1, 40):
        x, y = sb.step(J, h, x, y, a0, a0, 1.0, dt, sb.BSB)
        np.testing.assert_allclose(y, y0, rtol=0, atol=0)
        np.testing.assert_allclose(x, x0 + k * dt * a0 * y0, rtol=1e-12, atol=1e-15)
    M = np.array([[1.0 - (dt * a0) ** 2, dt * a0], [-dt * a0, 1.0]])
    x, y = x0.copy(), y0.copy()
    for k in range(1, 60):
        x, y = sb.step(J, h, x, y, 0.0, a0, 1.0, dt, sb.BSB)
        Mk = np.linalg.matrix_power(M, k)
        np.testing.assert_allclose(x, Mk[0, 0] * x0 + Mk[0, 1] * y0, rtol=1e-10, atol=1e-15)
        np.testing.assert_allclose(y, Mk[1, 0] * x0 + Mk[1, 1] * y0, rtol=1e-10, atol=1e-15)


def test_step_is_symplectic():
    """Symplectic Euler is a composition of two shears: the Jacobian of one step
    has determinant 1 (an explicit Euler step would not)."""
    q = random_qubo(6, 3, seed=2)
    J, h, _ = ising.to_ising(q)
    rng = np.random.default_rng(0)
    x = rng.uniform(-0.5, 0.5, 6)
    y = rng.uniform(-0.5, 0.5, 6)
    for variant in (sb.ASB, sb.BSB):
        def f(z):
            xn, yn = sb.step(J, h, z[:6], z[6:], 0.3, 1.0, 0.7, 0.1, variant)
            return np.concatenate([xn, yn])
        z = np.concatenate([x, y])
        eps = 1e-6
        Jac = np.stack([(f(z + eps * e) - f(z - eps * e)) / (2 * eps) for e in np.eye(12)], axis=1)
        assert np.linalg.det(Jac) == pytest.approx(1.0, abs=1e-6)


def test_hamiltonian_is_conserved():
    """With a(t) held fixed and a small dt, the trajectory keeps the Hamiltonian of
    Eq. 3-4 (aSB) or Eq. 7-8 (bSB inside the box) to O(dt); a wrong sign of any
    force term would make it drift."""
    q = random_qubo(10, 3, seed=4)
    J, h, _ = ising.to_ising(q)
    x, y = sb.init_state(2, 10, 4)
    x, y = x * 20, y * 20
    dt, a, a0, c0 = 1e-3, 0.4, 1.0, 0.3
    for variant in (sb.ASB, sb.BSB):
        H0 = sb.hamiltonian(J, h, x, y, a, a0, c0, variant)
        xx, yy = x.copy(), y.copy()
        drift = 0.0
        for _ in range(2000):
            xx, yy = sb.step(J, h, xx, yy, a, a0, c0, dt, variant)
            assert np.max(np.abs(xx)) < 1.0
            drift = max(drift, np.max(np.abs(sb.hamiltonian(J, h, xx, yy, a, a0, c0, variant) - H0)))
        assert drift < 5e-4 * max(1.0, np.max(np.abs(H0)))
        # the same trajectory with the momentum update using the wrong sign of the
        # coupling drifts far more (the check has teeth)
        xx, yy = x.copy(), y.copy()
        bad = 0.0
        for _ in range(2000):
            xx, yy = sb.step(-J, -h, xx, yy, a, a0, c0, dt, variant)
            bad = max(bad, np.max(np.abs(sb.hamiltonian(J, h, xx, yy, a, a0, c0, variant) - H0)))
        assert bad > 10 * drift


def test_field_equals_pinned_ancilla():
    """The field term c0 h_i equals a coupling J_{i,anc} = h_i to an extra spin
    whose position stays at +1."""
    import scipy.sparse as sp
    q = random_qubo(15, 4, seed=8)
    J, h, _ = ising.to_ising(q)
    n = q.n
    Ja = sp.bmat([[J, sp.csr_matrix(h[:, None])], [sp.csr_matrix(h[None, :]), None]]).tocsr()
    x, y = sb.init_state(3, n, 4)
    xa = np.vstack([x, np.ones((1, 4))])
    ya = np.vstack([y, np.zeros((1, 4))])
    for variant in (sb.BSB, sb.DSB, sb.ASB):
        xx, yy, xxa, yya = x.copy(), y.copy(), xa.copy(), ya.copy()
        for a_k in sb.linear_schedule(1.0, 200):
            xx, yy = sb.step(J, h, xx, yy, a_k, 1.0, 0.8, 0.3, variant)
            xxa, yya = sb.step(Ja, np.zeros(n + 1), xxa, yya, a_k, 1.0, 0.8, 0.3, variant)
            xxa[-1] = 1.0
            yya[-1] = 0.0
            np.testing.assert_allclose(xx, xxa[:-1], rtol=1e-13, atol=1e-13)


def test_dsb_equals_bsb_on_the_walls():
    """When every x_j is at a wall (+-1), sgn(x_j) = x_j, so one dSB step equals one bSB step."""
    q = random_qubo(30, 5, seed=6)
    J, h, _ = ising.to_ising(q)
    rng = np.random.default_rng(4)
    x = rng.choice([-1.0, 1.0], size=(30, 5))
    y = rng.uniform(-0.1, 0.1, size=(30, 5))
    xb, yb = sb.step(J, h, x, y, 0.2, 1.0, 0.5, 0.5, sb.BSB)
    xd, yd = sb.step(J, h, x, y, 0.2, 1.0, 0.5, 0.5, sb.DSB)
    np.testing.assert_array_equal(xb, xd)
    np.testing.assert_array_equal(yb, yd)


def test_init_state_range_and_determinism():
    x, y = sb.init_state(42, 100, 8)
    assert np.all(np.abs(x) <= 0.01) and np.all(np.abs(y) <= 0.01)
    assert np.all(x.astype(np.float32).astype(np.float64) == x)
    x2, _ = sb.init_state(42, 100, 8)
    np.testing.assert_array_equal(x, x2)
    x3, _ = sb.init_state(43, 100, 8)
    assert not np.array_equal(x, x3)
    assert abs(float(np.mean(x))) < 1e-3 and 0.004 < float(np.std(x)) < 0.0075


# ---------------------------------------------------------------- tracks
def test_truth_selection_scores_perfectly():
    """Selecting exactly the true triplets of clean, isolated tracks gives 100 %
    efficiency and purity (Eq. 18-19)."""
    seed, ev = _separated_seed(5, 0.5)
    p = qubo.BuildParams(dphi_slope=1.5e-3, dphi_margin=1.0, z0_max=100, kappa_max=2e-3,
                         dtheta_max=0.2, dkappa_max=5e-4)
    q = qubo.build_qubo(ev, p)
    T = np.array([1 if ev.particle[a] == ev.particle[b] == ev.particle[c] >= 0 else 0
                  for (a, b, c) in q.trip])
    trks, reco = tracks.assemble(q, T)
    assert len(trks) == 5 and all(len(t) == 10 for t in trks)
    tp, fp, fn, eff, pur = tracks.score(ev, reco)
    assert (tp, fp, fn, eff, pur) == (45, 0, 0, 1.0, 1.0)
    # nothing selected
    _, reco0 = tracks.assemble(q, np.zeros(q.n, int))
    assert tracks.score(ev, reco0) == (0, 0, 45, 0.0, 0.0)


def test_conflicting_doublets_are_removed_and_short_tracks_dropped():
    d = {(0, 1), (1, 2), (2, 3), (3, 4), (1, 5), (10, 11), (11, 12)}
    kept = tracks.resolve_conflicts(d)
    assert kept == {(0, 1), (2, 3), (3, 4), (10, 11), (11, 12)}
    assert tracks.chain(kept) == []          # 2-3-4 and 10-11-12 have 3 hits
    assert tracks.chain({(0, 1), (1, 2), (2, 3)}) == [[0, 1, 2, 3]]


def test_efficiency_and_purity_by_hand():
    """Eq. 18-19 on a hand-built event: efficiency = TP / (TP + FN) over the
    true doublets (hits of one particle on adjacent layers), purity = TP /
    (TP + FP) over the selected ones; the two differ, so a swap is caught."""
    from types import SimpleNamespace
    # particle 0 on layers 0-3, particle 1 on layers 0-3, particle 2 on layers
    # 0 and 2 (no adjacent pair), two noise hits
    ev = SimpleNamespace(particle=[0, 0, 0, 0, 1, 1, 1, 1, 2, 2, -1, -1],
                         layer=[0, 1, 2, 3, 0, 1, 2, 3, 0, 2, 1, 2])
    assert tracks.true_doublets(ev) == {(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (6, 7)}
    reco = {(0, 1), (1, 2), (2, 3), (10, 11)}
    assert tracks.score(ev, reco) == (3, 1, 3, 0.5, 0.75)
    reco = {(4, 5), (5, 6), (6, 7), (0, 1), (1, 2), (2, 3), (8, 9), (10, 11)}
    assert tracks.score(ev, reco) == (6, 2, 0, 1.0, 0.75)


# ---------------------------------------------------------------- TTT
def test_ttt_closed_forms():
    assert ttt.ttt_at(2.0, 1.0) == 2.0
    assert ttt.ttt_at(2.0, 0.0) == math.inf
    assert ttt.ttt_at(1.0, 0.5) == pytest.approx(math.log(0.01) / math.log(0.5))
    # p = 1 - 0.01^(1/4): four repetitions reach 99 %
    p = 1.0 - 0.01 ** 0.25
    assert ttt.ttt_at(3.0, p) == pytest.approx(12.0)
    assert ttt.target_energy(-100.0) == pytest.approx(-99.9)
    assert ttt.ttt([1.0, 2.0], [[0, 0, 0, 5], [0, 0, 0, 0]], 0.5) == pytest.approx(min(math.log(0.01) / math.log(0.25), 2.0))
    assert ttt.ttt([1.0], [[1.0, 2.0]], 0.5) is None
    # at or above 99 % one run suffices; a batch of R replicas succeeds if any does
    assert ttt.ttt_at(2.0, 0.995) == 2.0
    assert ttt.p_batch(0.5, 3) == pytest.approx(0.875)
    assert ttt.ttt([1.0], [[0, 5, 5, 5]], 0.5, replicas_per_run=4) == pytest.approx(
        math.log(0.01) / math.log(0.75 ** 4))


# ---------------------------------------------------------------- paper-exact weights
def test_impact_parameters_closed_forms():
    """Points on a circle of radius R centred at (X, 0): closest approach to the
    origin |X - R|; a straight r-z line through (r, z) pairs meets r = 0 at its
    intercept; collinear transverse points fall back to the point-line distance."""
    R, X = 800.0, 803.25
    pts = [(X + R * math.cos(t), R * math.sin(t)) for t in (2.9, 3.0, 3.1)]
    zs = [(r, 2.5 + 0.75 * r) for r in (32.0, 72.0, 116.0)]
    d0, z0 = qubo.impact_parameters(pts[0][0], pts[0][1], zs[0][1], zs[0][0], pts[1][0], pts[1][1],
                                    pts[2][0], pts[2][1], zs[2][1], zs[2][0])
    assert d0 == pytest.approx(abs(X - R), abs=1e-9)
    assert z0 == pytest.approx(2.5, abs=1e-12)
    d0, _ = qubo.impact_parameters(1.0, 3.0, 0.0, 1.0, 2.0, 3.0, 5.0, 3.0, 1.0, 2.0)
    assert d0 == pytest.approx(3.0, abs=1e-15)


def test_pair_consistency_matches_eq14_by_hand():
    t = (0, 1, 2, 2.0e-4, 0.03)
    u = (1, 2, 3, 1.5e-4, 0.01)
    assert qubo.pair_consistency(t, u) == pytest.approx(1.0 - 0.5 * (5e-5 + 0.03), abs=1e-15)


def test_paper_weights_on_clean_tracks():
    """Clean isolated tracks from the origin: consistent couplings are -S_ij
    (close to -1, inside (-1, -1 + dtheta_max/2]); the Eq. 15 bias sits near its
    z0 term, d0 being ~0 for tracks from the beam line."""
    seed, ev = _separated_seed(4, 0.6)
    p = qubo.BuildParams(dphi_slope=1.5e-3, dphi_margin=1.0, z0_max=100, kappa_max=2e-3,
                         dtheta_max=0.2, dkappa_max=5e-4, coupling_mode=1, bias_mode=1)
    q = qubo.build_qubo(ev, p)
    assert q.n == 32
    assert np.all((q.val < -0.9) & (q.val >= -1.0))
    for i in range(q.n):
        a, _, c = q.trip[i]
        qq, pt, eta, phi0, z0, rc = ev.truth[ev.particle[a]]
        # the straight r-z line through the truth helix at r_a and r_c, read at r = 0
        za = z0 + math.sinh(eta) * 2 * rc * math.asin(ev.r[a] / (2 * rc))
        zc = z0 + math.sinh(eta) * 2 * rc * math.asin(ev.r[c] / (2 * rc))
        z_line = za - ev.r[a] * (zc - za) / (ev.r[c] - ev.r[a])
        expect = 0.2 * (1.0 - math.exp(-abs(z_line) / 0.5))   # d0 = 0 for tracks from the origin
        assert q.quality[i] == pytest.approx(expect, abs=1e-6)


# ---------------------------------------------------------------- pins added for c0, bias, pruning, draws
def test_sigma_j_and_c0_closed_form():
    """Hand-built 4-variable QUBO with b_01 = b_12 = +1 (both triangles): J = -b/4
    has k = 4 off-diagonal entries of magnitude 1/4, so the RMS over the n(n-1)
    = 12 off-diagonal slots is sigma_J = (1/4) sqrt(4/12) and
    c0 = 0.5 / (sqrt(4) sigma_J) = sqrt(3). A mean-subtracted std, an n^2 or an
    nnz denominator, or one triangle only would each give another number."""
    from tests.inputs import QuboArrays
    q = QuboArrays(4, np.array([0, 1, 3, 4, 4], np.int32), np.array([1, 0, 2, 1], np.int32),
                   np.array([1.0, 1.0, 1.0, 1.0]), np.zeros(4))
    J, _, _ = ising.to_ising(q)
    assert ising.sigma_j(J, 4) == pytest.approx(0.25 * math.sqrt(4.0 / 12.0), rel=1e-15)
    assert ising.c0_auto(J, 4) == pytest.approx(math.sqrt(3.0), rel=1e-15)
    # one entry of magnitude v among n = 3 variables: sigma_J = v sqrt(2 / 6)
    q3 = QuboArrays(3, np.array([0, 1, 2, 2], np.int32), np.array([1, 0], np.int32),
                    np.array([-2.0, -2.0]), np.zeros(3))
    J3, _, _ = ising.to_ising(q3)
    assert ising.sigma_j(J3, 3) == pytest.approx(0.5 * math.sqrt(2.0 / 6.0), rel=1e-15)
    assert ising.c0_auto(J3, 3) == pytest.approx(0.5 / (math.sqrt(3.0) * 0.5 / math.sqrt(3.0)),
                                                rel=1e-15)


def test_default_bias_from_truth_curvature_and_angle():
    """Default linear term of Eq. 13 (triplet-quality reading): a_i = w_q (|kappa_i| /
    kappa_max + dtheta_i / dtheta_max) / 2, here computed from the generator's truth
    alone -- kappa = 1 / Rc of the helix, dtheta from the truth helix's r-z points --
    for unsmeared isolated tracks, with w_q = 1.7 and unequal cut scales so that a
    swapped kappa_max / dtheta_max, a missing 1/2 or a dropped w_q fails."""
    seed, ev = _separated_seed(4, 0.6)
    kmax, tmax, wq = 2e-3, 0.2, 1.7
    p = qubo.BuildParams(dphi_slope=1.5e-3, dphi_margin=1.0, z0_max=100, kappa_max=kmax,
                         dtheta_max=tmax, dkappa_max=5e-4, w_q=wq)
    q = qubo.build_qubo(ev, p)
    assert q.n == 32
    for i in range(q.n):
        a, b, c = q.trip[i]
        qq, pt, eta, phi0, z0, rc = ev.truth[ev.particle[a]]

        def zs(h):
            return math.sinh(eta) * 2 * rc * math.asin(ev.r[h] / (2 * rc))
        th1 = math.atan2(ev.r[b] - ev.r[a], zs(b) - zs(a))
        th2 = math.atan2(ev.r[c] - ev.r[b], zs(c) - zs(b))
        expect = wq * 0.5 * ((1.0 / rc) / kmax + abs(th2 - th1) / tmax)
        assert q.lin[i] == pytest.approx(expect, rel=1e-6)
        assert q.quality[i] == pytest.approx(expect / wq, rel=1e-6)


def _hand_event(tracks_spec):
    """Straight radial tracks (phi, first layer, n layers), z = 0.5 r; hits sorted."""
    radii = events.LAYER_RADII
    hits = []
    for t, (phi, l0, nl) in enumerate(tracks_spec):
        for l in range(l0, l0 + nl):
            hits.append((l, phi, 0.5 * radii[l], t))
    hits.sort(key=lambda h: (h[0], h[1]))
    ev = events.Event(layer=[], r=[], phi=[], z=[], x=[], y=[], particle=[], n_true=len(hits))
    for (l, phi, z, part) in hits:
        r = radii[l]
        ev.layer.append(l); ev.r.append(r); ev.phi.append(phi); ev.z.append(z)
        ev.x.append(r * math.cos(phi)); ev.y.append(r * math.sin(phi)); ev.particle.append(part)
    return ev


def test_pruning_keeps_only_five_hit_candidates():
    """Pruning rule (section "QUBO Generation and Track Finding"): a quadruplet
    must belong to a candidate of five or more hits. Three isolated straight
    tracks of 3, 4 and 5 hits: the 3-hit track's triplet is in no quadruplet and
    is always dropped; the 4-hit track's two triplets form one consistent pair
    with no consistent neighbour on either side and are dropped under the rule;
    the 5-hit track keeps its three triplets. Without the rule the 4-hit pair
    stays."""
    ev = _hand_event([(-2.0, 0, 3), (0.5, 2, 4), (2.5, 4, 5)])
    base = dict(dphi_slope=1e-3, dphi_margin=1.0, z0_max=100, kappa_max=2e-3, dtheta_max=0.2,
                dkappa_max=5e-4)
    q = qubo.build_qubo(ev, qubo.BuildParams(five_hit_rule=True, **base))
    parts = sorted(ev.particle[int(t[0])] for t in q.trip)
    assert parts == [2, 2, 2]
    assert len(q.col) == 4 and np.all(q.val == -1.0)
    q2 = qubo.build_qubo(ev, qubo.BuildParams(five_hit_rule=False, **base))
    parts2 = sorted(ev.particle[int(t[0])] for t in q2.trip)
    assert parts2 == [1, 1, 2, 2, 2]
    # the dropped triplets are exactly the ones whose pair has no consistent neighbour
    trip = qubo.build_triplets(ev, qubo.build_doublets(ev, qubo.BuildParams(**base)),
                               qubo.BuildParams(**base))
    assert len(trip) == 1 + 2 + 3


def test_track_parameter_draws_follow_the_recipe():
    """Distribution pins of the generator's draws over 2000 tracks (Kolmogorov-
    Smirnov against the stated laws, each also rejecting a plausible wrong law):
    1/pT ~ U[0.1, 1] GeV^-1 (not pT ~ U[1, 10]), eta ~ U(-1, 1), phi0 ~ U[0, 2 pi),
    z0 ~ N(0, 5 mm), q = +-1 with probability 1/2."""
    from scipy import stats
    ev = events.generate(2718, events.EventParams(n_tracks=2000, noise_frac=0.0))
    q = np.array([t[0] for t in ev.truth])
    pt = np.array([t[1] for t in ev.truth])
    eta = np.array([t[2] for t in ev.truth])
    phi0 = np.array([t[3] for t in ev.truth])
    z0 = np.array([t[4] for t in ev.truth])
    assert set(np.unique(q)) == {-1.0, 1.0} and abs(float(np.mean(q))) < 0.1
    assert stats.kstest(1.0 / pt, lambda v: stats.uniform.cdf(v, 0.1, 0.9)).pvalue > 1e-3
    assert stats.kstest(pt, lambda v: stats.uniform.cdf(v, 1.0, 9.0)).pvalue < 1e-6
    assert pt.min() >= 1.0 and pt.max() <= 10.0
    assert stats.kstest(eta, lambda v: stats.uniform.cdf(v, -1.0, 2.0)).pvalue > 1e-3
    assert stats.kstest(eta, lambda v: stats.uniform.cdf(v, 0.0, 1.0)).pvalue < 1e-6
    assert stats.kstest(phi0, lambda v: stats.uniform.cdf(v, 0.0, 2 * math.pi)).pvalue > 1e-3
    assert stats.kstest(phi0, lambda v: stats.uniform.cdf(v, -math.pi, 2 * math.pi)).pvalue < 1e-6
    assert stats.kstest(z0, lambda v: stats.norm.cdf(v / 5.0)).pvalue > 1e-3
    assert stats.kstest(z0, lambda v: stats.norm.cdf(v)).pvalue < 1e-6
