"""Simulated bifurcation time evolution (oracle side), FP64. Test infrastructure only.

Section "Simulated Bifurcation":
* aSB, Eq. 1-2:  dx/dt = a0 y,  dy/dt = -[x^2 + a0 - a(t)] x + c0 sum_j J_ij x_j
* bSB, Eq. 5-6:  dy/dt = -[a0 - a(t)] x + c0 sum_j J_ij x_j, with the fully
  inelastic wall: once |x_i| > 1, x_i <- sgn(x_i) and y_i <- 0 (Eq. 8).
* dSB, Eq. 9-10: as bSB but the coupling uses sgn(x_j) (Eq. 10), same wall.
* integration: symplectic Euler (all positions and momenta updated at once):
  the momentum is advanced with the old positions, then the position with
  the new momentum.

Readings where the paper is silent (each also listed in the design notes):
* the Ising field h enters the force as c0 h_i, i.e. as a coupling to an
  extra spin pinned at +1 (Eq. 2/6/10 print no field term);
* a(t): linear from 0 to a0 over the run, a_k = a0 k / (S - 1);
* wall test is strict (|x| > 1); sgn(0) = 0 inside the dSB product;
* initial x_i, y_i ~ U(-0.01, 0.01) drawn from Philox4x32-10 with counter
  (i, r, 3, event) and key = seed: word 0 gives x, word 1 gives y, as
  v = (w >> 8) - 2^23 and x = fp32(v) * fp32(fp32(0.01) * 2^-23).
"""
from dataclasses import dataclass

import numpy as np

from .philox import philox4x32_10, seed_key, PURPOSE_INIT

ASB, BSB, DSB = 0, 1, 2


def linear_schedule(a0, steps):
    """a_k = a0 k / (S - 1), k = 0..S-1 (a single step uses a = 0)."""
    if steps <= 1:
        return np.zeros(max(steps, 0))
    return np.array([a0 * k / (steps - 1) for k in range(steps)], dtype=np.float64)


def init_state(seed, n, R, event=0):
    """Initial (x, y), shape [n, R], FP32 values held in float64."""
    i = np.repeat(np.arange(n, dtype=np.uint64), R)
    r = np.tile(np.arange(R, dtype=np.uint64), n)
    k0, k1 = seed_key(seed)
    w0, w1, _, _ = philox4x32_10(i, r, np.full_like(i, PURPOSE_INIT),
                                 np.full_like(i, event), np.uint64(k0), np.uint64(k1))
    scale = np.float32(np.float32(0.01) * np.float32(2.0 ** -23))

    def conv(w):
        v = (w >> np.uint64(8)).astype(np.int64) - (1 << 23)
        return (v.astype(np.float32) * scale).astype(np.float64)

    return conv(w0).reshape(n, R), conv(w1).reshape(n, R)


def coupling(J, x, variant):
    """f = J g(x): g = identity (aSB, bSB, Eq. 2, 6) or sgn (dSB, Eq. 10)."""
    g = np.sign(x) if variant == DSB else x
    return J @ g


def step(J, h, x, y, a_k, a0, c0, dt, variant):
    """One symplectic-Euler step from (x, y); returns the new (x, y)."""
    f = coupling(J, x, variant)
    hh = h[:, None] if x.ndim == 2 else h
    force = -(a0 - a_k) * x + c0 * (f + hh)
    if variant == ASB:
        force = force - x ** 3
    y = y + dt * force
    x = x + dt * a0 * y
    if variant != ASB:
        hit = np.abs(x) > 1.0
        x = np.where(hit, np.sign(x), x)
        y = np.where(hit, 0.0, y)
    return x, y


@dataclass
class RunResult:
    x: np.ndarray
    y: np.ndarray
    trace: list


def run(J, h, x, y, sched, a0, c0, dt, variant, observe=None, every=0):
    """Advance len(sched) steps. ``observe(k, x, y)`` is called after step k when
    ``every`` > 0 and (k + 1) % every == 0; its results are collected in ``trace``."""
    trace = []
    for k, a_k in enumerate(sched):
        x, y = step(J, h, x, y, float(a_k), a0, c0, dt, variant)
        if every and (k + 1) % every == 0 and observe is not None:
            trace.append(observe(k, x, y))
    return RunResult(x, y, trace)


def hamiltonian(J, h, x, y, a, a0, c0, variant):
    """H of Eq. 3-4 (aSB) or Eq. 7-8 (bSB, inside the box), plus the field term
    -c0 h^T x of the force reading; per replica."""
    kin = 0.5 * a0 * np.sum(y * y, axis=0)
    pot = 0.5 * (a0 - a) * np.sum(x * x, axis=0) - 0.5 * c0 * np.sum(x * (J @ x), axis=0)
    pot = pot - c0 * (h @ x)
    if variant == ASB:
        pot = pot + 0.25 * np.sum(x ** 4, axis=0)
    return kin + pot


def step_rows(J, h, x, y, rows, a_k, a0, c0, dt, variant):
    """The step above for a subset of rows only (neighbours read from the full x);
    returns the new (x, y) of those rows."""
    rows = np.asarray(rows)
    g = np.sign(x) if variant == DSB else x
    f = J[rows] @ g
    xr, yr = x[rows], y[rows]
    force = -(a0 - a_k) * xr + c0 * (f + h[rows][:, None])
    if variant == ASB:
        force = force - xr ** 3
    yr = yr + dt * force
    xr = xr + dt * a0 * yr
    if variant != ASB:
        hit = np.abs(xr) > 1.0
        xr = np.where(hit, np.sign(xr), xr)
        yr = np.where(hit, 0.0, yr)
    return xr, yr


def prewall_x(J, h, x, y, a_k, a0, c0, dt, variant, rows=None):
    """Position after the momentum and position update but before the wall
    (used to recognise wall decisions that sit within rounding of |x| = 1)."""
    if rows is None:
        rows = np.arange(x.shape[0])
    g = np.sign(x) if variant == DSB else x
    xr, yr = x[rows], y[rows]
    force = -(a0 - a_k) * xr + c0 * (J[rows] @ g + h[rows][:, None])
    if variant == ASB:
        force = force - xr ** 3
    return xr + dt * a0 * (yr + dt * force)
