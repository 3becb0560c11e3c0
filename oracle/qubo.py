"""Triplet QUBO builder (oracle side): sections "QUBO Formulation" (Eq. 13)
and "QUBO Generation and Track Finding" (Eq. 16, 17 and the pruning rule).

Test infrastructure only. Plain loops; numpy is used only for element-wise
IEEE arithmetic (+ - * / sqrt, compares), never for transcendental functions.

Steps, in the paper's order:
1. doublets: hit pairs on consecutive layers that pass a phi window that
   grows with the radial gap, and a z-pointing cut on the origin;
2. triplets: two doublets sharing the middle hit, kept if Eq. 16 holds:
   holes H = 0 (layers l, l+1, l+2 only), |kappa| <= kappa_max, and
   dtheta <= dtheta_max.  kappa is the signed curvature [mm^-1] of the circle
   through the three transverse points (reading: the printed q/pT cut is
   taken as a curvature in mm^-1; 1 GeV at 2 T is 6e-4 mm^-1);
3. quadruplets: triplet pairs (a,b,c),(b,c,d) with |kappa_t - kappa_u| <=
   dkappa_max (Eq. 17, same unit reading);
4. pruning: a quadruplet must extend to a >= 5 hit candidate (it has a
   consistent predecessor or successor); triplets in no such quadruplet are
   dropped (done once);
5. Eq. 13 weights among the surviving triplets:
   b_ij = -1 for a consistent pair (the -S_ij of Eq. 14 replaced by -1),
   b_ij = +w_c for a conflict, i.e. two triplets that share a hit and start
   on the same or on adjacent layers but are not a consistent pair (they
   cannot both lie on one track), b_ij = 0 otherwise (no shared hit, or only
   the junction hit of (a,b,c),(c,d,e));
   a_i = w_q * quality_i, quality_i = (|kappa_i|/kappa_max +
   dtheta_i/dtheta_max) / 2 (reading of the bias weight as a triplet quality).

Paper-exact options:
* coupling_mode = 1: consistent pairs carry b_ij = -S_ij of Eq. 14,
  S_ij = (1 - (|kappa_i - kappa_j| + max(dtheta_i, dtheta_j)) / 2) / (1 + H_i + H_j)^2
  (H = 0: no holes are built), and a quadruplet also needs S_ij > s_min (Eq. 17);
* bias_mode = 1: quality_i follows Eq. 15 read with a decaying exponential,
  alpha (1 - exp(-|d0|/gamma)) + beta (1 - exp(-|z0|/lambda)), where d0 is the
  transverse distance of closest approach of the triplet's circle to the beam
  line and z0 the z of the triplet's r-z line at r = 0.

Triplet index order: lexicographic in (hit a, hit b, hit c).
Output CSR holds both triangles, ascending columns, no diagonal.
"""
import math
from dataclasses import dataclass

import numpy as np

from .events import TWO_PI

CLASS_CONSISTENT = 0
CLASS_CONFLICT = 1


@dataclass
class BuildParams:
    dphi_slope: float = 3.5e-4     # rad per mm of radial gap
    dphi_margin: float = 0.3       # mm, divided by the inner radius
    z0_max: float = 40.0           # mm, |z at r = 0| of the doublet line
    kappa_max: float = 8e-4        # mm^-1 (Eq. 16)
    dtheta_max: float = 0.1        # rad (Eq. 16)
    dkappa_max: float = 1e-4       # mm^-1 (Eq. 17)
    w_q: float = 1.0               # bias weight scale
    w_c: float = 1.0               # conflict weight scale
    five_hit_rule: bool = True
    coupling_mode: int = 0         # 0: b = -1 for consistent pairs; 1: b = -S_ij (Eq. 14)
    bias_mode: int = 0             # 0: curvature/angle quality; 1: Eq. 15 (d0, z0)
    s_min: float = 0.2             # Eq. 17 cut on S_ij (coupling_mode 1)
    alpha: float = 0.5             # Eq. 15 parameters
    beta: float = 0.2
    gamma: float = 1.0
    lam: float = 0.5


@dataclass
class Qubo:
    n: int
    rowptr: np.ndarray   # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]  (b_ij)
    lin: np.ndarray      # float64 [n]    (a_i)
    cls: np.ndarray      # int8 [nnz]     CLASS_CONSISTENT / CLASS_CONFLICT
    quality: np.ndarray  # float64 [n]
    trip: np.ndarray     # int32 [n, 3]   hit ids (a, b, c)
    kappa: np.ndarray    # float64 [n]
    dtheta: np.ndarray   # float64 [n]


def build_doublets(ev, p: BuildParams):
    """Doublets (h_in, h_out) on consecutive layers, lexicographic order."""
    layer = np.asarray(ev.layer)
    r = np.asarray(ev.r, dtype=np.float64)
    phi = np.asarray(ev.phi, dtype=np.float64)
    z = np.asarray(ev.z, dtype=np.float64)
    out = []
    nl = int(layer.max()) + 1 if len(layer) else 0
    for l in range(nl - 1):
        inner = np.nonzero(layer == l)[0]
        outer = np.nonzero(layer == l + 1)[0]
        if len(inner) == 0 or len(outer) == 0:
            continue
        for h in inner:
            dphi = phi[outer] - phi[h]
            dphi = dphi - TWO_PI * np.floor((dphi + math.pi) / TWO_PI)
            dr = r[outer] - r[h]
            win = p.dphi_slope * dr + p.dphi_margin / r[h]
            z0 = z[h] - r[h] * (z[outer] - z[h]) / dr
            ok = (np.abs(dphi) <= win) & (np.abs(z0) <= p.z0_max)
            for o in outer[ok]:
                out.append((int(h), int(o)))
    return out


def curvature(xa, ya, xb, yb, xc, yc):
    """Signed curvature of the circle through three points: 2 cross / (d_ab d_bc d_ac)."""
    dx1 = xb - xa
    dy1 = yb - ya
    dx2 = xc - xb
    dy2 = yc - yb
    dx3 = xc - xa
    dy3 = yc - ya
    cross = dx1 * dy2 - dy1 * dx2
    d1 = math.sqrt(dx1 * dx1 + dy1 * dy1)
    d2 = math.sqrt(dx2 * dx2 + dy2 * dy2)
    d3 = math.sqrt(dx3 * dx3 + dy3 * dy3)
    return 2.0 * cross / (d1 * d2 * d3)


def impact_parameters(xa, ya, za, ra, xb, yb, xc, yc, zc, rc):
    """(d0, z0) of a triplet: closest approach of the circle through the three
    transverse points to the origin, and the r = 0 intercept of the a-c line in r-z."""
    d = 2.0 * (xa * (yb - yc) + xb * (yc - ya) + xc * (ya - yb))
    z0 = za - ra * (zc - za) / (rc - ra)
    if d == 0.0:
        lx = xc - xa
        ly = yc - ya
        return abs(xa * yc - xc * ya) / math.sqrt(lx * lx + ly * ly), z0
    sa = xa * xa + ya * ya
    sb_ = xb * xb + yb * yb
    sc = xc * xc + yc * yc
    ux = (sa * (yb - yc) + sb_ * (yc - ya) + sc * (ya - yb)) / d
    uy = (sa * (xc - xb) + sb_ * (xa - xc) + sc * (xb - xa)) / d
    rad = math.sqrt((xa - ux) * (xa - ux) + (ya - uy) * (ya - uy))
    return abs(math.sqrt(ux * ux + uy * uy) - rad), z0


def pair_consistency(t, u):
    """S_ij of Eq. 14 with no holes: 1 - (|kappa_t - kappa_u| + max(dtheta_t, dtheta_u)) / 2."""
    return 1.0 - 0.5 * (abs(t[3] - u[3]) + max(t[4], u[4]))


def build_triplets(ev, doublets, p: BuildParams):
    """Triplets passing Eq. 16; list of (a, b, c, kappa, dtheta) sorted by (a, b, c)."""
    theta = {}
    for (h, o) in doublets:
        theta[(h, o)] = math.atan2(ev.r[o] - ev.r[h], ev.z[o] - ev.z[h])
    incoming = {}
    outgoing = {}
    for (h, o) in doublets:
        outgoing.setdefault(h, []).append(o)
        incoming.setdefault(o, []).append(h)
    trip = []
    for b in sorted(incoming):
        if b not in outgoing:
            continue
        for a in incoming[b]:
            for c in outgoing[b]:
                kap = curvature(ev.x[a], ev.y[a], ev.x[b], ev.y[b], ev.x[c], ev.y[c])
                dth = abs(theta[(b, c)] - theta[(a, b)])
                if abs(kap) <= p.kappa_max and dth <= p.dtheta_max:
                    trip.append((a, b, c, kap, dth))
    trip.sort(key=lambda t: (t[0], t[1], t[2]))
    return trip


def classify_pairs(ev, trip, p: BuildParams):
    """All triplet pairs with a non-zero Eq. 13 weight: dict (i, j) -> class, i != j."""
    by_hit = {}
    for i, t in enumerate(trip):
        for h in t[:3]:
            by_hit.setdefault(h, []).append(i)
    pairs = {}
    for i, t in enumerate(trip):
        lt = ev.layer[t[0]]
        cand = set()
        for h in t[:3]:
            cand.update(by_hit[h])
        cand.discard(i)
        for j in cand:
            u = trip[j]
            lu = ev.layer[u[0]]
            if abs(lu - lt) >= 2:
                continue                      # at most the junction hit: compatible
            if lu == lt + 1 and t[1] == u[0] and t[2] == u[1]:
                ok = abs(t[3] - u[3]) <= p.dkappa_max
            elif lu == lt - 1 and u[1] == t[0] and u[2] == t[1]:
                ok = abs(u[3] - t[3]) <= p.dkappa_max
            else:
                ok = False
            if ok and p.coupling_mode == 1:
                ok = pair_consistency(t, u) > p.s_min
            pairs[(i, j)] = CLASS_CONSISTENT if ok else CLASS_CONFLICT
    return pairs


def prune(ev, trip, pairs, p: BuildParams):
    """Indices of triplets that survive the quadruplet rule, ascending."""
    succ = {}
    pred = {}
    for (i, j), c in pairs.items():
        if c != CLASS_CONSISTENT:
            continue
        if ev.layer[trip[j][0]] == ev.layer[trip[i][0]] + 1:
            succ.setdefault(i, []).append(j)
            pred.setdefault(j, []).append(i)
    keep = set()
    for i, js in succ.items():
        for j in js:
            if (not p.five_hit_rule) or (i in pred) or (j in succ):
                keep.add(i)
                keep.add(j)
    return sorted(keep)


def build_qubo(ev, p: BuildParams = BuildParams()):
    """Event -> Qubo (Eq. 13) with the cuts of Eq. 16, 17 and the pruning rule."""
    doublets = build_doublets(ev, p)
    trip = build_triplets(ev, doublets, p)
    pairs = classify_pairs(ev, trip, p)
    keep = prune(ev, trip, pairs, p)
    new_index = {old: k for k, old in enumerate(keep)}
    n = len(keep)
    rows = [[] for _ in range(n)]
    for (i, j), c in pairs.items():
        if i in new_index and j in new_index:
            if c == CLASS_CONSISTENT:
                v = -pair_consistency(trip[i], trip[j]) if p.coupling_mode == 1 else -1.0
            else:
                v = p.w_c
            rows[new_index[i]].append((new_index[j], v, c))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    col, val, cls = [], [], []
    for i in range(n):
        rows[i].sort()
        for (j, v, c) in rows[i]:
            col.append(j)
            val.append(v)
            cls.append(c)
        rowptr[i + 1] = len(col)
    quality = np.zeros(n)
    lin = np.zeros(n)
    kap = np.zeros(n)
    dth = np.zeros(n)
    tri = np.zeros((n, 3), dtype=np.int32)
    for k, old in enumerate(keep):
        a, b, c, kk, dd = trip[old]
        if p.bias_mode == 1:
            d0, z0 = impact_parameters(ev.x[a], ev.y[a], ev.z[a], ev.r[a], ev.x[b], ev.y[b],
                                       ev.x[c], ev.y[c], ev.z[c], ev.r[c])
            quality[k] = (p.alpha * (1.0 - math.exp(-abs(d0) / p.gamma)) +
                          p.beta * (1.0 - math.exp(-abs(z0) / p.lam)))
        else:
            quality[k] = 0.5 * (abs(kk) / p.kappa_max + dd / p.dtheta_max)
        lin[k] = p.w_q * quality[k]
        kap[k] = kk
        dth[k] = dd
        tri[k] = (a, b, c)
    return Qubo(n, rowptr, np.asarray(col, dtype=np.int32), np.asarray(val, dtype=np.float64),
                lin, np.asarray(cls, dtype=np.int8), quality, tri, kap, dth)
