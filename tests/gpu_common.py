"""Helpers shared by the GPU parity tests (no arithmetic of the method)."""
import functools

import numpy as np
import scipy.sparse as sp

import paper_2402_14718_gb300 as sb
from paper_2402_14718_gb300.workloads import WORKLOADS
from oracle import events as oev
from oracle import ising
from oracle import qubo as oq


def oracle_params(cuts):
    kw = dict(cuts)
    kw["five_hit_rule"] = bool(kw["five_hit_rule"])
    return oq.BuildParams(**kw)


@functools.lru_cache(maxsize=None)
def workload_qubos(name):
    """(product event, product qubo, oracle event, oracle qubo) of a named workload."""
    w = WORKLOADS[name]
    ev_c = sb.sb_event_generate(w["seed"], sb.event_params(n_tracks=w["n_tracks"],
                                                            noise_frac=w["noise_frac"]))
    qc = sb.sb_qubo_build(ev_c, sb.build_params(**w["cuts"]))
    ev_o = oev.generate(w["seed"], oev.EventParams(n_tracks=w["n_tracks"],
                                                  noise_frac=w["noise_frac"]))
    qo = oq.build_qubo(ev_o, oracle_params(w["cuts"]))
    return ev_c, qc, ev_o, qo


def oracle_c0(qo):
    """c0 = 0.5 / (sqrt(N) sigma_J) computed by the oracle from its own QUBO;
    both sides of a parity test take this value (the library's own c0 is
    compared with it separately)."""
    J = ising.to_ising(qo)[0]
    return ising.c0_auto(J, qo.n)


def max_rel(a, ref):
    """max |a - ref| / max |ref| (scale-normalised error of one state array)."""
    scale = max(float(np.max(np.abs(ref))), 1e-30)
    return float(np.max(np.abs(np.asarray(a, np.float64) - ref))) / scale


def compare_step(xg, yg, xo, yo, xpre, tol=1e-5):
    """One-step parity with wall near-ties excluded: where the oracle's pre-wall
    |x| is within 1e-5 of 1 the two sides may take different wall decisions."""
    tie = np.abs(np.abs(xpre) - 1.0) < 1e-5
    keep = ~tie
    assert tie.mean() < 1e-3
    ex = max_rel(np.where(keep, xg, 0.0), np.where(keep, xo, 0.0))
    ey = max_rel(np.where(keep, yg, 0.0), np.where(keep, yo, 0.0))
    assert ex <= tol, ex
    assert ey <= tol, ey
    return ex, ey


def compare_step_elementwise(J, h, x0, y0, a_k, a0, c0, dt, variant, xg, yg, xo, yo, xpre,
                             rows=None, tol=1e-5):
    """Element-wise bar of one FP32 step: |gpu - oracle| <= tol * S per element,
    where S is the magnitude of the terms that form that element (FP32
    rounding is relative to it, not to the element's own value, which may
    cancel to ~0):
      S_y = |y| + dt (|(a0 - a_k) x| + |x|^3 [aSB] + c0 (sum_j |J_ij| |g(x_j)| + |h_i|)),
      S_x = |x| + dt a0 S_y,
    g = id (aSB, bSB) or sgn (dSB). Wall near-ties are excluded as in
    compare_step. Returns the worst ratios (x, y)."""
    x0 = np.asarray(x0, np.float64)
    y0 = np.asarray(y0, np.float64)
    g = np.abs(np.sign(x0)) if variant == 2 else np.abs(x0)
    Jabs = abs(J) if sp.issparse(J) else np.abs(J)
    sj = np.asarray(Jabs @ g)
    hb = np.abs(np.asarray(h, np.float64))[:, None]
    if rows is not None:
        x0, y0, sj, hb = x0[rows], y0[rows], sj[rows], hb[rows]
    sy = np.abs(y0) + dt * (abs(a0 - a_k) * np.abs(x0) + c0 * (sj + hb))
    if variant == 0:
        sy = sy + dt * np.abs(x0) ** 3
    sx = np.abs(x0) + dt * a0 * sy
    keep = np.abs(np.abs(xpre) - 1.0) >= 1e-5
    rx = np.where(keep, np.abs(np.asarray(xg, np.float64) - xo) / sx, 0.0)
    ry = np.where(keep, np.abs(np.asarray(yg, np.float64) - yo) / sy, 0.0)
    ex, ey = float(np.max(rx)), float(np.max(ry))
    assert ex <= tol, ex
    assert ey <= tol, ey
    return ex, ey
