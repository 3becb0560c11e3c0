"""Reverse-mode gradient of the relaxed bSB energy (oracle side, FP64).
Test infrastructure only.

Forward: the bSB steps of section "Simulated Bifurcation" (Eq. 5-8) with the
field reading of ``oracle.sb``; per step k
  y~ = y_k + dt (-(a0 - a_k) x_k + c0 (J x_k + h)),  x~ = x_k + dt a0 y~,
  m_k = |x~| > 1,  x_{k+1} = m ? sgn(x~) : x~,  y_{k+1} = m ? 0 : y~.
Loss: L = (1/R) sum_r E(x_S,r), E(x) = -(1/2) x^T J x - h^T x (offset excluded).
The wall is differentiated as the piecewise map it is: where m = 1 the new
position is a constant +-1 and the momentum 0, so no adjoint flows through.

QUBO weight scales: b_ij = -1 (consistent) or +w_c (conflict), a_i = w_q q_i,
so J = -b/4 and h = -(a/2 + sum_j b/4) are affine in (w_q, w_c):
  dJ_ij/dw_c = -1/4 on conflict entries, dh_i/dw_c = -n_conf_i / 4,
  dh_i/dw_q = -q_i / 2.
c0 is an independent input here (no automatic c0 in the gradient path).
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """Class-tagged QUBO: rowptr/col CSR, cls per entry (0 consistent, 1 conflict), quality per row."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    cls: np.ndarray
    quality: np.ndarray


def weights(p: Problem, w_q, w_c):
    """(J scipy CSR, h, C conflict adjacency CSR, n_conf) for the given scales."""
    b = np.where(p.cls == 0, -1.0, w_c)
    a = w_q * p.quality
    J = sp.csr_matrix((-b / 4.0, p.col, p.rowptr), shape=(p.n, p.n))
    C = sp.csr_matrix(((p.cls == 1).astype(np.float64), p.col, p.rowptr), shape=(p.n, p.n))
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    bsum = np.bincount(rows, weights=b, minlength=p.n)
    h = -(a / 2.0 + bsum / 4.0)
    n_conf = np.asarray(C.sum(axis=1)).ravel()
    return J, h, C, n_conf


def forward(J, h, x, y, sched, a0, c0, dt):
    """bSB forward keeping what the reverse sweep needs; returns (xs, yts, ms, loss)."""
    R = x.shape[1]
    xs, yts, ms = [x], [], []
    for a_k in sched:
        yt = y + dt * (-(a0 - a_k) * x + c0 * (J @ x + h[:, None]))
        xt = x + dt * a0 * yt
        m = np.abs(xt) > 1.0
        x = np.where(m, np.sign(xt), xt)
        y = np.where(m, 0.0, yt)
        xs.append(x)
        yts.append(yt)
        ms.append(m)
    loss = float(np.sum(-0.5 * x * (J @ x) - h[:, None] * x)) / R
    return xs, yts, ms, loss


def loss_only(p, x, y, sched, a0, c0, dt, w_q, w_c):
    J, h, _, _ = weights(p, w_q, w_c)
    return forward(J, h, x, y, sched, a0, c0, dt)[3]


def masks(p, x, y, sched, a0, c0, dt, w_q, w_c):
    J, h, _, _ = weights(p, w_q, w_c)
    return np.stack(forward(J, h, x, y, sched, a0, c0, dt)[2])


def gradient(p: Problem, x0, y0, sched, a0, c0, dt, w_q, w_c):
    """Returns (loss, dict(dt, c0, w_q, w_c, sched[S]))."""
    J, h, C, n_conf = weights(p, w_q, w_c)
    R = x0.shape[1]
    xs, yts, ms, loss = forward(J, h, x0, y0, sched, a0, c0, dt)
    xS = xs[-1]
    lx = (-(J @ xS) - h[:, None]) / R
    ly = np.zeros_like(lx)
    gh = -np.sum(xS, axis=1) / R
    g_wc = float(np.sum(xS * (C @ xS))) / (8.0 * R)
    g_dt = g_c0 = 0.0
    g_a = np.zeros(len(sched))
    for k in range(len(sched) - 1, -1, -1):
        keep = ~ms[k]
        lxt = np.where(keep, lx, 0.0)
        lyt = np.where(keep, ly, 0.0) + dt * a0 * lxt
        x = xs[k]
        f = J @ x
        F = -(a0 - sched[k]) * x + c0 * (f + h[:, None])
        g_dt += float(np.sum(lyt * F) + np.sum(lxt * a0 * yts[k]))
        g_c0 += float(np.sum(lyt * dt * (f + h[:, None])))
        g_a[k] = float(np.sum(lyt * dt * x))
        gh += dt * c0 * np.sum(lyt, axis=1)
        g_wc += float(np.sum(dt * c0 * lyt * (-0.25) * (C @ x)))
        lx = lxt - dt * (a0 - sched[k]) * lyt + dt * c0 * (J @ lyt)
        ly = lyt
    g_wq = float(np.sum(gh * (-p.quality / 2.0)))
    g_wc += float(np.sum(gh * (-n_conf / 4.0)))
    return loss, {"dt": g_dt, "c0": g_c0, "w_q": g_wq, "w_c": g_wc, "sched": g_a}
