// Triplet QUBO builder: sections "QUBO Formulation" (Eq. 13) and "QUBO
// Generation and Track Finding" (Eq. 16, 17 and the pruning rule).
//
// Compiled with -ffp-contract=off -fno-builtin: each cut is evaluated with
// plain IEEE double operations in the written order, so the CSR it produces
// is identical, bit for bit, to the one of the FP64 oracle.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <new>
#include <utility>

#include "host_internal.h"
#include "../guard.h"

namespace {

const double kTwoPi = 2.0 * M_PI;

struct Doublet {
  int32_t in, out;
  double theta;  // atan2(r_out - r_in, z_out - z_in): polar angle of the segment
};

struct Triplet {
  int32_t a, b, c;
  double kappa, dtheta;
};

// S_ij of Eq. 14 without holes
double pair_consistency(const Triplet& t, const Triplet& u) {
  return 1.0 - 0.5 * (fabs(t.kappa - u.kappa) + std::max(t.dtheta, u.dtheta));
}

// Signed curvature of the circle through three transverse points:
// 2 * cross(b - a, c - b) / (|b - a| |c - b| |c - a|); > 0 counter-clockwise.
double curvature(double xa, double ya, double xb, double yb, double xc, double yc) {
  double dx1 = xb - xa;
  double dy1 = yb - ya;
  double dx2 = xc - xb;
  double dy2 = yc - yb;
  double dx3 = xc - xa;
  double dy3 = yc - ya;
  double cross = dx1 * dy2 - dy1 * dx2;
  double d1 = sqrt(dx1 * dx1 + dy1 * dy1);
  double d2 = sqrt(dx2 * dx2 + dy2 * dy2);
  double d3 = sqrt(dx3 * dx3 + dy3 * dy3);
  return 2.0 * cross / (d1 * d2 * d3);
}

// (d0, z0) of a triplet: closest approach of the circle through the three
// transverse points to the origin, and the r = 0 intercept of the a-c line in r-z.
void impact_parameters(double xa, double ya, double za, double ra, double xb, double yb,
                       double xc, double yc, double zc, double rc, double* d0, double* z0) {
  double d = 2.0 * (xa * (yb - yc) + xb * (yc - ya) + xc * (ya - yb));
  *z0 = za - ra * (zc - za) / (rc - ra);
  if (d == 0.0) {
    double lx = xc - xa;
    double ly = yc - ya;
    *d0 = fabs(xa * yc - xc * ya) / sqrt(lx * lx + ly * ly);
    return;
  }
  double sa = xa * xa + ya * ya;
  double sb = xb * xb + yb * yb;
  double sc = xc * xc + yc * yc;
  double ux = (sa * (yb - yc) + sb * (yc - ya) + sc * (ya - yb)) / d;
  double uy = (sa * (xc - xb) + sb * (xa - xc) + sc * (xb - xa)) / d;
  double rad = sqrt((xa - ux) * (xa - ux) + (ya - uy) * (ya - uy));
  *d0 = fabs(sqrt(ux * ux + uy * uy) - rad);
}

enum : int8_t { kConsistent = 0, kConflict = 1 };

}  // namespace

extern "C" void sb_build_params_default(sb_build_params* p) {
  if (!p) return;
  p->dphi_slope = 3.5e-4;
  p->dphi_margin = 0.3;
  p->z0_max = 40.0;
  p->kappa_max = 8e-4;
  p->dtheta_max = 0.1;
  p->dkappa_max = 1e-4;
  p->w_q = 1.0;
  p->w_c = 1.0;
  p->five_hit_rule = 1;
  p->coupling_mode = 0;
  p->bias_mode = 0;
  p->s_min = 0.2;
  p->alpha = 0.5;
  p->beta = 0.2;
  p->gamma = 1.0;
  p->lambda = 0.5;
}

extern "C" sb_status sb_qubo_build(const sb_event* ev, const sb_build_params* p, sb_qubo** out) {
  return sbh::guarded("sb_qubo_build", [&]() -> sb_status {
    if (!ev || !p || !out) {
      sbh::set_error("sb_qubo_build: null argument");
      return SB_ERR_ARG;
    }
    if ((p->coupling_mode != 0 && p->coupling_mode != 1) || (p->bias_mode != 0 && p->bias_mode != 1) ||
        (p->bias_mode == 1 && !(p->gamma > 0.0 && p->lambda > 0.0))) {
      sbh::set_error("sb_qubo_build: coupling_mode / bias_mode must be 0 or 1, gamma and lambda > 0");
      return SB_ERR_ARG;
    }
    *out = nullptr;
    const int32_t nh = (int32_t)ev->layer.size();
    int nl = 0;
    for (int32_t h = 0; h < nh; ++h) nl = std::max(nl, ev->layer[h] + 1);

    // hit ids per layer (hits are sorted by layer, so each layer is a contiguous range)
    std::vector<int32_t> lstart(nl + 1, 0);
    for (int32_t h = 0; h < nh; ++h) lstart[ev->layer[h] + 1]++;
    for (int l = 0; l < nl; ++l) lstart[l + 1] += lstart[l];

    // 1. doublets, lexicographic in (in, out)
    std::vector<Doublet> dbl;
    for (int l = 0; l + 1 < nl; ++l) {
      for (int32_t h = lstart[l]; h < lstart[l + 1]; ++h) {
        const double ph = ev->phi[h], rh = ev->r[h], zh = ev->z[h];
        for (int32_t o = lstart[l + 1]; o < lstart[l + 2]; ++o) {
          double dphi = ev->phi[o] - ph;
          dphi = dphi - kTwoPi * floor((dphi + M_PI) / kTwoPi);
          double dr = ev->r[o] - rh;
          double win = p->dphi_slope * dr + p->dphi_margin / rh;
          double z0 = zh - rh * (ev->z[o] - zh) / dr;
          if (fabs(dphi) <= win && fabs(z0) <= p->z0_max)
            dbl.push_back(Doublet{h, o, atan2(ev->r[o] - rh, ev->z[o] - zh)});
        }
      }
    }

    // 2. triplets (Eq. 16)
    std::vector<std::vector<int32_t>> incoming(nh), outgoing(nh);  // doublet indices
    for (int32_t d = 0; d < (int32_t)dbl.size(); ++d) {
      outgoing[dbl[d].in].push_back(d);
      incoming[dbl[d].out].push_back(d);
    }
    std::vector<Triplet> trip;
    for (int32_t b = 0; b < nh; ++b) {
      for (int32_t di : incoming[b]) {
        const int32_t a = dbl[di].in;
        for (int32_t dj : outgoing[b]) {
          const int32_t c = dbl[dj].out;
          double kap = curvature(ev->x[a], ev->y[a], ev->x[b], ev->y[b], ev->x[c], ev->y[c]);
          double dth = fabs(dbl[dj].theta - dbl[di].theta);
          if (fabs(kap) <= p->kappa_max && dth <= p->dtheta_max)
            trip.push_back(Triplet{a, b, c, kap, dth});
        }
      }
    }
    std::sort(trip.begin(), trip.end(), [](const Triplet& s, const Triplet& t) {
      if (s.a != t.a) return s.a < t.a;
      if (s.b != t.b) return s.b < t.b;
      return s.c < t.c;
  });
  const int32_t nt = (int32_t)trip.size();

  // 3. pairs sharing a hit: consistent (Eq. 17) or conflicting
  std::vector<std::vector<int32_t>> by_hit(nh);
  for (int32_t i = 0; i < nt; ++i) {
    by_hit[trip[i].a].push_back(i);
    by_hit[trip[i].b].push_back(i);
    by_hit[trip[i].c].push_back(i);
  }
  struct Pair {
    int32_t i, j;
    int8_t cls;
  };
  std::vector<Pair> pairs;
  std::vector<int32_t> cand;
  for (int32_t i = 0; i < nt; ++i) {
    const Triplet& t = trip[i];
    const int lt = ev->layer[t.a];
    cand.clear();
    for (int32_t h : {t.a, t.b, t.c}) cand.insert(cand.end(), by_hit[h].begin(), by_hit[h].end());
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    for (int32_t j : cand) {
      if (j == i) continue;
      const Triplet& u = trip[j];
      const int lu = ev->layer[u.a];
      if (abs(lu - lt) >= 2) continue;  // at most the junction hit: compatible
      bool ok;
      if (lu == lt + 1 && t.b == u.a && t.c == u.b)
        ok = fabs(t.kappa - u.kappa) <= p->dkappa_max;
      else if (lu == lt - 1 && u.b == t.a && u.c == t.b)
        ok = fabs(u.kappa - t.kappa) <= p->dkappa_max;
      else
        ok = false;
      if (ok && p->coupling_mode == 1) ok = pair_consistency(t, u) > p->s_min;
      pairs.push_back(Pair{i, j, ok ? kConsistent : kConflict});
    }
  }

  // 4. pruning: keep quadruplets that extend to >= 5 hits
  std::vector<char> has_succ(nt, 0), has_pred(nt, 0), keep(nt, 0);
  for (const Pair& pr : pairs)
    if (pr.cls == kConsistent && ev->layer[trip[pr.j].a] == ev->layer[trip[pr.i].a] + 1) {
      has_succ[pr.i] = 1;
      has_pred[pr.j] = 1;
    }
  for (const Pair& pr : pairs)
    if (pr.cls == kConsistent && ev->layer[trip[pr.j].a] == ev->layer[trip[pr.i].a] + 1)
      if (!p->five_hit_rule || has_pred[pr.i] || has_succ[pr.j]) keep[pr.i] = keep[pr.j] = 1;
  std::vector<int32_t> new_index(nt, -1);
  int32_t n = 0;
  for (int32_t i = 0; i < nt; ++i)
    if (keep[i]) new_index[i] = n++;

  // 5. Eq. 13 weights, CSR over the survivors (pairs are already in (i, j) order)
  sb_qubo* q = new (std::nothrow) sb_qubo;
  if (!q) return SB_ERR_OOM;
  q->n = n;
  q->w_c = p->w_c;
  q->n_hits = nh;
  q->rowptr.assign(n + 1, 0);
  for (const Pair& pr : pairs) {
    const int32_t ni = new_index[pr.i], nj = new_index[pr.j];
    if (ni < 0 || nj < 0) continue;
    q->col.push_back(nj);
    double v = p->w_c;
    if (pr.cls == kConsistent)
      v = p->coupling_mode == 1 ? -pair_consistency(trip[pr.i], trip[pr.j]) : -1.0;
    q->val.push_back(v);
    q->cls.push_back(pr.cls);
    q->rowptr[ni + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) q->rowptr[i + 1] += q->rowptr[i];
  q->lin.resize(n);
  q->quality.resize(n);
  q->kappa.resize(n);
  q->dtheta.resize(n);
  q->trip.resize((size_t)3 * n);
  for (int32_t i = 0; i < nt; ++i) {
    const int32_t k = new_index[i];
    if (k < 0) continue;
    const Triplet& t = trip[i];
    if (p->bias_mode == 1) {
      double d0, z0;
      impact_parameters(ev->x[t.a], ev->y[t.a], ev->z[t.a], ev->r[t.a], ev->x[t.b], ev->y[t.b],
                        ev->x[t.c], ev->y[t.c], ev->z[t.c], ev->r[t.c], &d0, &z0);
      q->quality[k] = p->alpha * (1.0 - exp(-fabs(d0) / p->gamma)) +
                      p->beta * (1.0 - exp(-fabs(z0) / p->lambda));
    } else {
      q->quality[k] = 0.5 * (fabs(t.kappa) / p->kappa_max + t.dtheta / p->dtheta_max);
    }
    q->lin[k] = p->w_q * q->quality[k];
    q->kappa[k] = t.kappa;
    q->dtheta[k] = t.dtheta;
    q->trip[3 * (size_t)k] = t.a;
    q->trip[3 * (size_t)k + 1] = t.b;
    q->trip[3 * (size_t)k + 2] = t.c;
  }
  if ((int64_t)q->col.size() > (int64_t)0x7FFFFFFF) {
    delete q;
    sbh::set_error("sb_qubo_build: more than 2^31 - 1 couplings");
    return SB_ERR_ARG;
  }
  *out = q;
  return SB_OK;
  });
}

extern "C" sb_status sb_qubo_sizes(const sb_qubo* q, int32_t* n, int64_t* nnz) {
  if (!q) {
    sbh::set_error("sb_qubo_sizes: null qubo");
    return SB_ERR_ARG;
  }
  if (n) *n = q->n;
  if (nnz) *nnz = (int64_t)q->col.size();
  return SB_OK;
}

extern "C" sb_status sb_qubo_arrays(const sb_qubo* q, int32_t* rowptr, int32_t* col, double* val,
                                    double* lin, int8_t* cls, double* quality, int32_t* trip,
                                    double* kappa, double* dtheta) {
  if (!q) {
    sbh::set_error("sb_qubo_arrays: null qubo");
    return SB_ERR_ARG;
  }
  if (rowptr) std::copy(q->rowptr.begin(), q->rowptr.end(), rowptr);
  if (col) std::copy(q->col.begin(), q->col.end(), col);
  if (val) std::copy(q->val.begin(), q->val.end(), val);
  if (lin) std::copy(q->lin.begin(), q->lin.end(), lin);
  if (cls) std::copy(q->cls.begin(), q->cls.end(), cls);
  if (quality) std::copy(q->quality.begin(), q->quality.end(), quality);
  if (trip) std::copy(q->trip.begin(), q->trip.end(), trip);
  if (kappa) std::copy(q->kappa.begin(), q->kappa.end(), kappa);
  if (dtheta) std::copy(q->dtheta.begin(), q->dtheta.end(), dtheta);
  return SB_OK;
}

// The conflict part of Eq. 13 in factored form (reading of "any conflict": two
// triplets sharing a hit conflict when they start on the same or adjacent
// layers). A triplet holding hit h at position p starts on layer(h) - p, so
// two triplets sharing h at positions p, p' start |p - p'| layers apart: the
// group of (h, p) couples to the groups (h, p') with |p - p'| <= 1, weight w_c.
extern "C" sb_status sb_qubo_factor(const sb_qubo* q, int32_t* member, uint8_t* couple, double* w,
                                    int32_t* n_ids) {
  if (!q || !member || !couple || !w || !n_ids) {
    sbh::set_error("sb_qubo_factor: null argument");
    return SB_ERR_ARG;
  }
  std::copy(q->trip.begin(), q->trip.end(), member);
  for (int p = 0; p < 3; ++p)
    for (int p2 = 0; p2 < 3; ++p2) couple[3 * p + p2] = (p - p2 <= 1 && p2 - p <= 1) ? 1 : 0;
  *w = q->w_c;
  *n_ids = std::max<int32_t>(q->n_hits, 1);
  return SB_OK;
}

extern "C" void sb_qubo_destroy(sb_qubo* q) { delete q; }
