// Synthetic barrel events -- the stand-in for the TrackML events of section
// "Dataset": helical tracks in a uniform solenoid field crossing ten barrel
// cylinders, Gaussian measurement smear and uniform noise hits.
//
// Compiled with -ffp-contract=off -fno-builtin so that every floating-point
// operation is a plain IEEE double operation or a libm call in the written
// order (the FP64 oracle recomputes the same events bit for bit).
#include <math.h>

#include <algorithm>
#include <new>

#include "../philox.h"
#include "host_internal.h"
#include "../guard.h"

namespace {

const double kTwoPi = 2.0 * M_PI;

struct Draw {
  double u0, u1;
};

Draw draw(uint64_t seed, uint32_t purpose, uint32_t obj, uint32_t var) {
  sbk::U32x4 w = sbk::philox4x32_10(obj, var, purpose, 0u, (uint32_t)(seed & 0xFFFFFFFFu),
                                    (uint32_t)(seed >> 32));
  Draw d;
  d.u0 = sbk::uniform01(w.v[0], w.v[1]);
  d.u1 = sbk::uniform01(w.v[2], w.v[3]);
  return d;
}

// Box-Muller from one counter block.
double gauss(uint64_t seed, uint32_t purpose, uint32_t obj, uint32_t var) {
  Draw d = draw(seed, purpose, obj, var);
  return sqrt(-2.0 * log(1.0 - d.u0)) * cos(kTwoPi * d.u1);
}

double wrap_phi(double phi) { return phi - kTwoPi * floor((phi + M_PI) / kTwoPi); }

struct RawHit {
  int32_t layer;
  double phi, z;
  int32_t particle;
  int64_t gen;
};

}  // namespace

extern "C" void sb_event_params_default(sb_event_params* p) {
  if (!p) return;
  static const double radii[10] = {32.0, 72.0, 116.0, 172.0, 260.0,
                                   360.0, 500.0, 660.0, 820.0, 1000.0};
  p->n_tracks = 100;
  p->n_layers = 10;
  for (int l = 0; l < 16; ++l) p->radii[l] = l < 10 ? radii[l] : 0.0;
  p->noise_frac = 0.1;
  p->bz = 2.0;
  p->inv_pt_min = 0.1;
  p->inv_pt_max = 1.0;
  p->eta_max = 1.0;
  p->z0_sigma = 5.0;
  p->smear_rphi = 0.1;
  p->smear_z = 0.1;
}

extern "C" sb_status sb_event_generate(uint64_t seed, const sb_event_params* p, sb_event** out) {
  return sbh::guarded("sb_event_generate", [&]() -> sb_status {
    if (!p || !out) {
      sbh::set_error("sb_event_generate: null argument");
      return SB_ERR_ARG;
    }
    *out = nullptr;
    const int nl = p->n_layers;
    if (nl < 1 || nl > 16 || p->n_tracks < 0 || p->n_tracks > 10000000 || !(p->noise_frac >= 0.0) ||
        !(p->bz > 0.0) || !(p->inv_pt_min > 0.0) || !(p->inv_pt_max >= p->inv_pt_min)) {
      sbh::set_error("sb_event_generate: parameters out of range");
      return SB_ERR_ARG;
    }
    for (int l = 0; l < nl; ++l) {
      // every track must reach every layer: r < 2 Rc for the lowest pT
      double rc_min = (1000.0 * (1.0 / p->inv_pt_max)) / (0.3 * p->bz);
      if (!(p->radii[l] > 0.0) || (l && !(p->radii[l] > p->radii[l - 1])) ||
          !(p->radii[l] < 2.0 * rc_min)) {
        sbh::set_error("sb_event_generate: layer radii must ascend and stay below 2 Rc(min pT)");
        return SB_ERR_ARG;
      }
    }
    sb_event* ev = new (std::nothrow) sb_event;
    if (!ev) return SB_ERR_OOM;
    std::vector<RawHit> raw;
    raw.reserve((size_t)p->n_tracks * nl);
    for (int32_t t = 0; t < p->n_tracks; ++t) {
      const uint32_t P = sbk::kPurposeTrack, T = (uint32_t)t;
      double uq = draw(seed, P, T, 0).u0;
      double q = uq < 0.5 ? 1.0 : -1.0;
      double ui = draw(seed, P, T, 1).u0;
      double inv_pt = p->inv_pt_min + (p->inv_pt_max - p->inv_pt_min) * ui;
      double ue = draw(seed, P, T, 2).u0;
      double eta = -p->eta_max + 2.0 * p->eta_max * ue;
      double up = draw(seed, P, T, 3).u0;
      double phi0 = kTwoPi * up;
      double z0 = p->z0_sigma * gauss(seed, P, T, 4);
      double pt = 1.0 / inv_pt;
      double rc = (1000.0 * pt) / (0.3 * p->bz);
      double sh = sinh(eta);
      for (int l = 0; l < nl; ++l) {
        double r = p->radii[l];
        double a = asin(r / (2.0 * rc));
        double phi = phi0 - q * a;
        double z = z0 + (2.0 * rc * a) * sh;
        phi = phi + (p->smear_rphi * gauss(seed, P, T, 5u + (uint32_t)l)) / r;
        z = z + p->smear_z * gauss(seed, P, T, 5u + (uint32_t)nl + (uint32_t)l);
        raw.push_back(RawHit{l, wrap_phi(phi), z, t, (int64_t)t * nl + l});
      }
    }
    const int64_t n_true = (int64_t)raw.size();
    double zmin[16], zmax[16];
    for (int l = 0; l < 16; ++l) {
      zmin[l] = INFINITY;
      zmax[l] = -INFINITY;
    }
    for (const RawHit& h : raw) {
      zmin[h.layer] = std::min(zmin[h.layer], h.z);
      zmax[h.layer] = std::max(zmax[h.layer], h.z);
    }
    int64_t n_noise = n_true ? (int64_t)floor(p->noise_frac * (double)n_true + 0.5) : 0;
    for (int64_t k = 0; k < n_noise; ++k) {
      const uint32_t P = sbk::kPurposeNoise, K = (uint32_t)k;
      double ul = draw(seed, P, K, 0).u0;
      int l = std::min((int)floor(ul * nl), nl - 1);
      double up = draw(seed, P, K, 1).u0;
      double phi = -M_PI + kTwoPi * up;
      double uz = draw(seed, P, K, 2).u0;
      double z = zmin[l] + (zmax[l] - zmin[l]) * uz;
      raw.push_back(RawHit{l, wrap_phi(phi), z, -1, n_true + k});
    }
    std::sort(raw.begin(), raw.end(), [](const RawHit& a, const RawHit& b) {
      if (a.layer != b.layer) return a.layer < b.layer;
      if (a.phi != b.phi) return a.phi < b.phi;
      return a.gen < b.gen;
  });
  const size_t nh = raw.size();
  ev->layer.resize(nh);
  ev->r.resize(nh);
  ev->phi.resize(nh);
  ev->z.resize(nh);
  ev->x.resize(nh);
  ev->y.resize(nh);
  ev->particle.resize(nh);
  for (size_t k = 0; k < nh; ++k) {
    const RawHit& h = raw[k];
    double r = p->radii[h.layer];
    ev->layer[k] = h.layer;
    ev->r[k] = r;
    ev->phi[k] = h.phi;
    ev->z[k] = h.z;
    ev->x[k] = r * cos(h.phi);
    ev->y[k] = r * sin(h.phi);
    ev->particle[k] = h.particle;
  }
  ev->n_true = (int32_t)n_true;
  *out = ev;
  return SB_OK;
  });
}

extern "C" int32_t sb_event_num_hits(const sb_event* ev) { return ev ? (int32_t)ev->layer.size() : 0; }
extern "C" int32_t sb_event_num_true(const sb_event* ev) { return ev ? ev->n_true : 0; }

extern "C" sb_status sb_event_hits(const sb_event* ev, int32_t* layer, double* r, double* phi,
                                   double* z, double* x, double* y, int32_t* particle) {
  if (!ev) {
    sbh::set_error("sb_event_hits: null event");
    return SB_ERR_ARG;
  }
  const size_t n = ev->layer.size();
  if (layer) std::copy(ev->layer.begin(), ev->layer.end(), layer);
  if (r) std::copy(ev->r.begin(), ev->r.end(), r);
  if (phi) std::copy(ev->phi.begin(), ev->phi.end(), phi);
  if (z) std::copy(ev->z.begin(), ev->z.end(), z);
  if (x) std::copy(ev->x.begin(), ev->x.end(), x);
  if (y) std::copy(ev->y.begin(), ev->y.end(), y);
  if (particle) std::copy(ev->particle.begin(), ev->particle.end(), particle);
  (void)n;
  return SB_OK;
}

extern "C" void sb_event_destroy(sb_event* ev) { delete ev; }
