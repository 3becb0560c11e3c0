// Triplet-QUBO builder on the GPU: the host builder's steps (sections "QUBO
// Formulation", Eq. 13, and "QUBO Generation and Track Finding", Eq. 16, 17,
// pruning) as count / scan / write passes over hits, doublets and triplets.
//
// Compiled with -fmad=false: every +, -, *, /, sqrt is the single IEEE FP64
// operation the host builder performs, in the same order, so the cut
// decisions and values agree with the host bit for bit except where they go
// through atan2 (segment angles) or exp (Eq. 15 bias), whose device and host
// implementations may differ in the last place.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../host/host_internal.h"
#include "../guard.h"

namespace {

constexpr int kB = 256;
constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * kPi;

int grid_of(long long n) {
  long long g = (n + kB - 1) / kB;
  if (g < 1) g = 1;
  if (g > 65535LL * 16) g = 65535LL * 16;
  return (int)g;
}

// ------------------------------------------------------------------ exclusive scan (int64)
__global__ void k_scan_block(const long long* in, long long* out, long long* sums, long long n) {
  __shared__ long long sh[1024];
  const long long base = (long long)blockIdx.x * 1024;
  const int t = threadIdx.x;
  long long v0 = base + 2 * t < n ? in[base + 2 * t] : 0;
  long long v1 = base + 2 * t + 1 < n ? in[base + 2 * t + 1] : 0;
  sh[2 * t] = v0;
  sh[2 * t + 1] = v1;
  for (int off = 1; off < 1024; off <<= 1) {
    __syncthreads();
    const int i = (t + 1) * off * 2 - 1;
    if (i < 1024) sh[i] += sh[i - off];
  }
  __syncthreads();
  if (t == 0) {
    if (sums) sums[blockIdx.x] = sh[1023];
    sh[1023] = 0;
  }
  for (int off = 512; off >= 1; off >>= 1) {
    __syncthreads();
    const int i = (t + 1) * off * 2 - 1;
    if (i < 1024) {
      const long long tmp = sh[i - off];
      sh[i - off] = sh[i];
      sh[i] += tmp;
    }
  }
  __syncthreads();
  if (base + 2 * t < n) out[base + 2 * t] = sh[2 * t];
  if (base + 2 * t + 1 < n) out[base + 2 * t + 1] = sh[2 * t + 1];
}

__global__ void k_scan_add(long long* out, const long long* add, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += add[i / 1024];
}

// out = exclusive scan of in (n values); returns the total in *total (host)
cudaError_t exclusive_scan(const long long* in, long long* out, long long n, long long* total,
                           cudaStream_t s) {
  if (n <= 0) {
    *total = 0;
    return cudaSuccess;
  }
  const long long nb = (n + 1023) / 1024;
  long long* sums = nullptr;
  long long* ssum = nullptr;
  cudaError_t e = cudaMalloc(&sums, nb * sizeof(long long));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&ssum, nb * sizeof(long long));
  if (e != cudaSuccess) {
    cudaFree(sums);
    return e;
  }
  k_scan_block<<<(unsigned)nb, 512, 0, s>>>(in, out, sums, n);
  e = cudaGetLastError();
  long long sub_total = 0;
  if (e == cudaSuccess && nb > 1) {
    e = exclusive_scan(sums, ssum, nb, &sub_total, s);
    if (e == cudaSuccess) {
      k_scan_add<<<(unsigned)((n + kB - 1) / kB), kB, 0, s>>>(out, ssum, n);
      e = cudaGetLastError();
    }
  }
  long long last_in = 0, last_out = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&last_in, in + n - 1, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&last_out, out + n - 1, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *total = last_in + last_out;
  cudaFree(sums);
  cudaFree(ssum);
  return e;
}

// ------------------------------------------------------------------ hits
struct Hits {
  const int32_t* layer;
  const double *r, *phi, *z, *x, *y;
  const int32_t* lstart;  // [nl + 1]
  int32_t nh, nl;
};

struct Cuts {
  double dphi_slope, dphi_margin, z0_max, kappa_max, dtheta_max, dkappa_max, w_q, w_c;
  int five_hit_rule, coupling_mode, bias_mode;
  double s_min, alpha, beta, gamma, lambda;
};

__device__ __forceinline__ bool doublet_pass(const Hits& H, const Cuts& p, int h, int o) {
  double dphi = H.phi[o] - H.phi[h];
  dphi = dphi - kTwoPi * floor((dphi + kPi) / kTwoPi);
  const double dr = H.r[o] - H.r[h];
  const double win = p.dphi_slope * dr + p.dphi_margin / H.r[h];
  const double z0 = H.z[h] - H.r[h] * (H.z[o] - H.z[h]) / dr;
  return fabs(dphi) <= win && fabs(z0) <= p.z0_max;
}

// first index in [lo, hi) with phi >= v
__device__ __forceinline__ int lower_phi(const double* phi, int lo, int hi, double v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (phi[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// first index in [lo, hi) with phi > v
__device__ __forceinline__ int upper_phi(const double* phi, int lo, int hi, double v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (phi[mid] <= v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Candidate outer hits of inner hit h as ascending, disjoint index ranges. The
// exact test accepts o only if phi_o lies within win of phi_h modulo 2 pi, so
// with the window widened by 1e-6 rad (far above the rounding of the wrap) the
// candidates are: phi in [hi - 2pi] from -pi (wrap from above: lowest
// indices), the main window, and phi from lo + 2pi up to pi (wrap from below:
// highest indices). Outer hits share the layer radius, so win is one number.
__device__ __forceinline__ int window_ranges(const Hits& H, const Cuts& p, int h, int* r0,
                                             int* r1) {
  const int l = H.layer[h];
  const int o0 = H.lstart[l + 1], o1 = H.lstart[l + 2];
  if (o0 >= o1) return 0;
  const double w = p.dphi_slope * (H.r[o0] - H.r[h]) + p.dphi_margin / H.r[h] + 1e-6;
  if (w >= kPi) {
    r0[0] = o0;
    r1[0] = o1;
    return 1;
  }
  const double lo = H.phi[h] - w, hi = H.phi[h] + w;
  int s0[3] = {o0, 0, 0}, s1[3] = {o0, 0, 0};
  if (hi > kPi) s1[0] = upper_phi(H.phi, o0, o1, hi - kTwoPi);
  s0[1] = lower_phi(H.phi, o0, o1, lo);
  s1[1] = upper_phi(H.phi, o0, o1, hi);
  s0[2] = o1;
  s1[2] = o1;
  if (lo < -kPi) s0[2] = lower_phi(H.phi, o0, o1, lo + kTwoPi);
  int n = 0, prev_end = o0;
  for (int k = 0; k < 3; ++k) {
    const int x0 = s0[k] < prev_end ? prev_end : s0[k];
    const int x1 = s1[k];
    if (x0 < x1) {
      r0[n] = x0;
      r1[n] = x1;
      ++n;
      prev_end = x1;
    }
  }
  return n;
}

__global__ void k_doublet_count(Hits H, Cuts p, long long* cnt) {
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < H.nh; h += gridDim.x * blockDim.x) {
    long long c = 0;
    if (H.layer[h] + 1 < H.nl) {
      int r0[3], r1[3];
      const int nr = window_ranges(H, p, h, r0, r1);
      for (int k = 0; k < nr; ++k)
        for (int o = r0[k]; o < r1[k]; ++o) c += doublet_pass(H, p, h, o) ? 1 : 0;
    }
    cnt[h] = c;
  }
}

__global__ void k_doublet_write(Hits H, Cuts p, const long long* off, int32_t* d_out,
                                double* d_theta) {
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < H.nh; h += gridDim.x * blockDim.x) {
    if (H.layer[h] + 1 >= H.nl) continue;
    long long w = off[h];
    int r0[3], r1[3];
    const int nr = window_ranges(H, p, h, r0, r1);
    for (int k = 0; k < nr; ++k)
      for (int o = r0[k]; o < r1[k]; ++o)
        if (doublet_pass(H, p, h, o)) {
          d_out[w] = o;
          d_theta[w] = atan2(H.r[o] - H.r[h], H.z[o] - H.z[h]);
          ++w;
        }
  }
}

// ------------------------------------------------------------------ triplets
__device__ __forceinline__ double curvature(double xa, double ya, double xb, double yb,
                                            double xc, double yc) {
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

// doublets of inner hit h: [doff[h], doff[h+1]) with outer hits d_out[] ascending
template <bool WRITE>
__global__ void k_triplets(Hits H, Cuts p, const long long* doff, const int32_t* d_out,
                           const double* d_theta, const long long* toff, long long* tcnt,
                           int32_t* ta, int32_t* tb, int32_t* tc, double* tk, double* tdth) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < H.nh; a += gridDim.x * blockDim.x) {
    long long c = 0, w = WRITE ? toff[a] : 0;
    for (long long d1 = doff[a]; d1 < doff[a + 1]; ++d1) {
      const int b = d_out[d1];
      for (long long d2 = doff[b]; d2 < doff[b + 1]; ++d2) {
        const int cc = d_out[d2];
        const double kap = curvature(H.x[a], H.y[a], H.x[b], H.y[b], H.x[cc], H.y[cc]);
        const double dth = fabs(d_theta[d2] - d_theta[d1]);
        if (fabs(kap) <= p.kappa_max && dth <= p.dtheta_max) {
          if (WRITE) {
            ta[w] = a;
            tb[w] = b;
            tc[w] = cc;
            tk[w] = kap;
            tdth[w] = dth;
            ++w;
          } else {
            ++c;
          }
        }
      }
    }
    if (!WRITE) tcnt[a] = c;
  }
}

// ------------------------------------------------------------------ hit -> triplet lists
__global__ void k_incidence_count(const int32_t* ta, const int32_t* tb, const int32_t* tc,
                                  long long nt, unsigned long long* hcnt) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
       t += (long long)gridDim.x * blockDim.x) {
    atomicAdd(hcnt + ta[t], 1ull);
    atomicAdd(hcnt + tb[t], 1ull);
    atomicAdd(hcnt + tc[t], 1ull);
  }
}

__global__ void k_incidence_fill(const int32_t* ta, const int32_t* tb, const int32_t* tc,
                                 long long nt, const long long* hoff, unsigned long long* hfill,
                                 int32_t* list) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
       t += (long long)gridDim.x * blockDim.x) {
    const int32_t hs[3] = {ta[t], tb[t], tc[t]};
    for (int k = 0; k < 3; ++k) {
      const unsigned long long slot = atomicAdd(hfill + hs[k], 1ull);
      list[hoff[hs[k]] + (long long)slot] = (int32_t)t;
    }
  }
}

// each hit's list in ascending triplet order (insertion sort; lists are short)
__global__ void k_incidence_sort(const long long* hoff, int32_t nh, int32_t* list) {
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
    const long long b = hoff[h], e = hoff[h + 1];
    for (long long i = b + 1; i < e; ++i) {
      const int32_t v = list[i];
      long long j = i - 1;
      while (j >= b && list[j] > v) {
        list[j + 1] = list[j];
        --j;
      }
      list[j + 1] = v;
    }
  }
}

// ------------------------------------------------------------------ pairs
struct Trip {
  const int32_t *a, *b, *c;
  const double *k, *dth;
  long long n;
};

__device__ __forceinline__ double pair_consistency(const Trip& T, long long i, long long j) {
  return 1.0 - 0.5 * (fabs(T.k[i] - T.k[j]) + fmax(T.dth[i], T.dth[j]));
}

// class of (i, j): 0 consistent, 1 conflict, -1 no coupling (same rule as the host)
__device__ __forceinline__ int pair_class(const Hits& H, const Cuts& p, const Trip& T,
                                          long long i, long long j) {
  const int lt = H.layer[T.a[i]], lu = H.layer[T.a[j]];
  if (abs(lu - lt) >= 2) return -1;
  bool ok;
  if (lu == lt + 1 && T.b[i] == T.a[j] && T.c[i] == T.b[j])
    ok = fabs(T.k[i] - T.k[j]) <= p.dkappa_max;
  else if (lu == lt - 1 && T.b[j] == T.a[i] && T.c[j] == T.b[i])
    ok = fabs(T.k[j] - T.k[i]) <= p.dkappa_max;
  else
    ok = false;
  if (ok && p.coupling_mode == 1) ok = pair_consistency(T, i, j) > p.s_min;
  return ok ? 0 : 1;
}

// Walk the union of the three ascending incidence lists of triplet i (each
// partner once, in ascending order), calling f(j) for j != i.
template <typename F>
__device__ __forceinline__ void for_each_partner(const Trip& T, const long long* hoff,
                                                 const int32_t* list, long long i, F f) {
  const int32_t hs[3] = {T.a[i], T.b[i], T.c[i]};
  long long pos[3], end[3];
  for (int k = 0; k < 3; ++k) {
    pos[k] = hoff[hs[k]];
    end[k] = hoff[hs[k] + 1];
  }
  long long last = -1;
  while (true) {
    long long best = -1;
    for (int k = 0; k < 3; ++k)
      if (pos[k] < end[k]) {
        const long long v = list[pos[k]];
        if (best < 0 || v < best) best = v;
      }
    if (best < 0) break;
    for (int k = 0; k < 3; ++k)
      if (pos[k] < end[k] && list[pos[k]] == best) ++pos[k];
    if (best != last && best != i) f(best);
    last = best;
  }
}

__global__ void k_pairs(Hits H, Cuts p, Trip T, const long long* hoff, const int32_t* list,
                        const long long* poff, long long* pcnt, int32_t* pj, int8_t* pcls) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.n;
       i += (long long)gridDim.x * blockDim.x) {
    long long c = 0;
    long long w = poff ? poff[i] : 0;
    for_each_partner(T, hoff, list, i, [&](long long j) {
      const int cls = pair_class(H, p, T, i, j);
      if (cls < 0) return;
      if (poff) {
        pj[w] = (int32_t)j;
        pcls[w] = (int8_t)cls;
        ++w;
      } else {
        ++c;
      }
    });
    if (!poff) pcnt[i] = c;
  }
}

// has_succ / has_pred over consistent pairs (i -> j one layer out)
__global__ void k_links(Hits H, Trip T, const long long* poff, const int32_t* pj,
                        const int8_t* pcls, uint8_t* has_succ, uint8_t* has_pred) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.n;
       i += (long long)gridDim.x * blockDim.x) {
    for (long long q = poff[i]; q < poff[i + 1]; ++q) {
      const long long j = pj[q];
      if (pcls[q] == 0 && H.layer[T.a[j]] == H.layer[T.a[i]] + 1) {
        has_succ[i] = 1;
        has_pred[j] = 1;
      }
    }
  }
}

__global__ void k_keep(Hits H, Cuts p, Trip T, const long long* poff, const int32_t* pj,
                       const int8_t* pcls, const uint8_t* has_succ, const uint8_t* has_pred,
                       uint8_t* keep) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.n;
       i += (long long)gridDim.x * blockDim.x) {
    for (long long q = poff[i]; q < poff[i + 1]; ++q) {
      const long long j = pj[q];
      if (pcls[q] == 0 && H.layer[T.a[j]] == H.layer[T.a[i]] + 1)
        if (!p.five_hit_rule || has_pred[i] || has_succ[j]) {
          keep[i] = 1;
          keep[j] = 1;
        }
    }
  }
}

__global__ void k_u8_to_ll(const uint8_t* in, long long* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// final CSR rows of the kept triplets
__global__ void k_rows(Trip T, const long long* poff, const int32_t* pj, const uint8_t* keep,
                       const long long* newidx, long long* rcnt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.n;
       i += (long long)gridDim.x * blockDim.x) {
    if (!keep[i]) continue;
    long long c = 0;
    for (long long q = poff[i]; q < poff[i + 1]; ++q) c += keep[pj[q]] ? 1 : 0;
    rcnt[newidx[i]] = c;
  }
}

__global__ void k_rows_write(Hits H, Cuts p, Trip T, const long long* poff, const int32_t* pj,
                             const int8_t* pcls, const uint8_t* keep, const long long* newidx,
                             const long long* roff, int32_t* col, double* val, int8_t* cls,
                             double* quality, double* lin, int32_t* trip, double* kappa,
                             double* dtheta) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < T.n;
       i += (long long)gridDim.x * blockDim.x) {
    if (!keep[i]) continue;
    const long long k = newidx[i];
    long long w = roff[k];
    for (long long q = poff[i]; q < poff[i + 1]; ++q) {
      const long long j = pj[q];
      if (!keep[j]) continue;
      col[w] = (int32_t)newidx[j];
      double v = p.w_c;
      if (pcls[q] == 0) v = p.coupling_mode == 1 ? -pair_consistency(T, i, j) : -1.0;
      val[w] = v;
      cls[w] = pcls[q];
      ++w;
    }
    double qv;
    if (p.bias_mode == 1) {
      const int a = T.a[i], b = T.b[i], c = T.c[i];
      const double xa = H.x[a], ya = H.y[a], za = H.z[a], ra = H.r[a];
      const double xb = H.x[b], yb = H.y[b];
      const double xc = H.x[c], yc = H.y[c], zc = H.z[c], rc = H.r[c];
      double d = 2.0 * (xa * (yb - yc) + xb * (yc - ya) + xc * (ya - yb));
      double z0 = za - ra * (zc - za) / (rc - ra);
      double d0;
      if (d == 0.0) {
        double lx = xc - xa;
        double ly = yc - ya;
        d0 = fabs(xa * yc - xc * ya) / sqrt(lx * lx + ly * ly);
      } else {
        double sa = xa * xa + ya * ya;
        double sb = xb * xb + yb * yb;
        double sc = xc * xc + yc * yc;
        double ux = (sa * (yb - yc) + sb * (yc - ya) + sc * (ya - yb)) / d;
        double uy = (sa * (xc - xb) + sb * (xa - xc) + sc * (xb - xa)) / d;
        double rad = sqrt((xa - ux) * (xa - ux) + (ya - uy) * (ya - uy));
        d0 = fabs(sqrt(ux * ux + uy * uy) - rad);
      }
      qv = p.alpha * (1.0 - exp(-fabs(d0) / p.gamma)) + p.beta * (1.0 - exp(-fabs(z0) / p.lambda));
    } else {
      qv = 0.5 * (fabs(T.k[i]) / p.kappa_max + T.dth[i] / p.dtheta_max);
    }
    quality[k] = qv;
    lin[k] = p.w_q * qv;
    trip[3 * k] = T.a[i];
    trip[3 * k + 1] = T.b[i];
    trip[3 * k + 2] = T.c[i];
    kappa[k] = T.k[i];
    dtheta[k] = T.dth[i];
  }
}

// ------------------------------------------------------------------ device buffers
struct Pool {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T* get(long long count) {
    if (err != cudaSuccess) return nullptr;
    void* p = nullptr;
    err = cudaMalloc(&p, (size_t)std::max<long long>(count, 1) * sizeof(T));
    if (err != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Pool() {
    for (void* p : ptrs) cudaFree(p);
  }
};

}  // namespace

extern "C" sb_status sb_qubo_build_device(const sb_event* ev, const sb_build_params* bp,
                                          sb_qubo** out, double* out_device_ms, void* stream) {
  return sbh::guarded("sb_qubo_build_device", [&]() -> sb_status {
    if (!ev || !bp || !out) {
      sbh::set_error("sb_qubo_build_device: null argument");
      return SB_ERR_ARG;
    }
    *out = nullptr;
    if ((bp->coupling_mode != 0 && bp->coupling_mode != 1) ||
        (bp->bias_mode != 0 && bp->bias_mode != 1) ||
        (bp->bias_mode == 1 && !(bp->gamma > 0.0 && bp->lambda > 0.0))) {
      sbh::set_error("sb_qubo_build_device: coupling_mode / bias_mode must be 0 or 1");
      return SB_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t nh = (int32_t)ev->layer.size();
    int nl = 0;
    for (int32_t h = 0; h < nh; ++h) nl = std::max(nl, ev->layer[h] + 1);
    std::vector<int32_t> lstart(nl + 2, 0);
    for (int32_t h = 0; h < nh; ++h) lstart[ev->layer[h] + 1]++;
    for (int l = 0; l < nl; ++l) lstart[l + 1] += lstart[l];
    lstart[nl + 1] = lstart[nl];
    Pool P;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto fail = [&](cudaError_t e) {
      cudaGetLastError();  // clear a non-sticky error (allocation) before returning
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      sbh::set_error(std::string("sb_qubo_build_device: ") + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? SB_ERR_OOM : SB_ERR_CUDA;
    };
#define SB_B(call)                           \
    do {                                       \
      cudaError_t e_ = (call);                 \
      if (e_ != cudaSuccess) return fail(e_);  \
    } while (0)
    Hits H;
    int32_t* d_layer = P.get<int32_t>(nh);
    double* d_r = P.get<double>(nh);
    double* d_phi = P.get<double>(nh);
    double* d_z = P.get<double>(nh);
    double* d_x = P.get<double>(nh);
    double* d_y = P.get<double>(nh);
    int32_t* d_ls = P.get<int32_t>(nl + 2);
    SB_B(P.err);
    if (nh) {
      SB_B(cudaMemcpyAsync(d_layer, ev->layer.data(), nh * 4, cudaMemcpyHostToDevice, s));
      SB_B(cudaMemcpyAsync(d_r, ev->r.data(), nh * 8, cudaMemcpyHostToDevice, s));
      SB_B(cudaMemcpyAsync(d_phi, ev->phi.data(), nh * 8, cudaMemcpyHostToDevice, s));
      SB_B(cudaMemcpyAsync(d_z, ev->z.data(), nh * 8, cudaMemcpyHostToDevice, s));
      SB_B(cudaMemcpyAsync(d_x, ev->x.data(), nh * 8, cudaMemcpyHostToDevice, s));
      SB_B(cudaMemcpyAsync(d_y, ev->y.data(), nh * 8, cudaMemcpyHostToDevice, s));
    }
    SB_B(cudaMemcpyAsync(d_ls, lstart.data(), (nl + 2) * 4, cudaMemcpyHostToDevice, s));
    H.layer = d_layer;
    H.r = d_r;
    H.phi = d_phi;
    H.z = d_z;
    H.x = d_x;
    H.y = d_y;
    H.lstart = d_ls;
    H.nh = nh;
    H.nl = nl;
    Cuts p;
    p.dphi_slope = bp->dphi_slope;
    p.dphi_margin = bp->dphi_margin;
    p.z0_max = bp->z0_max;
    p.kappa_max = bp->kappa_max;
    p.dtheta_max = bp->dtheta_max;
    p.dkappa_max = bp->dkappa_max;
    p.w_q = bp->w_q;
    p.w_c = bp->w_c;
    p.five_hit_rule = bp->five_hit_rule;
    p.coupling_mode = bp->coupling_mode;
    p.bias_mode = bp->bias_mode;
    p.s_min = bp->s_min;
    p.alpha = bp->alpha;
    p.beta = bp->beta;
    p.gamma = bp->gamma;
    p.lambda = bp->lambda;
    SB_B(cudaEventRecord(e0, s));
    // 1. doublets
    long long* dcnt = P.get<long long>(nh + 1);
    long long* doff = P.get<long long>(nh + 1);
    SB_B(P.err);
    SB_B(cudaMemsetAsync(dcnt, 0, (nh + 1) * 8, s));
    k_doublet_count<<<grid_of(nh), kB, 0, s>>>(H, p, dcnt);
    SB_B(cudaGetLastError());
    long long nd = 0;
    SB_B(exclusive_scan(dcnt, doff, nh + 1, &nd, s));
    int32_t* d_out = P.get<int32_t>(nd);
    double* d_theta = P.get<double>(nd);
    SB_B(P.err);
    k_doublet_write<<<grid_of(nh), kB, 0, s>>>(H, p, doff, d_out, d_theta);
    SB_B(cudaGetLastError());
    // 2. triplets, lexicographic by construction (a, then b, then c ascending)
    long long* tcnt = P.get<long long>(nh + 1);
    long long* toff = P.get<long long>(nh + 1);
    SB_B(P.err);
    SB_B(cudaMemsetAsync(tcnt, 0, (nh + 1) * 8, s));
    k_triplets<false><<<grid_of(nh), kB, 0, s>>>(H, p, doff, d_out, d_theta, nullptr, tcnt, nullptr,
                                                 nullptr, nullptr, nullptr, nullptr);
    SB_B(cudaGetLastError());
    long long nt = 0;
    SB_B(exclusive_scan(tcnt, toff, nh + 1, &nt, s));
    if (nt >= 0x7FFFFFFFLL) return fail(cudaErrorInvalidValue);
    int32_t* ta = P.get<int32_t>(nt);
    int32_t* tb = P.get<int32_t>(nt);
    int32_t* tc = P.get<int32_t>(nt);
    double* tk = P.get<double>(nt);
    double* tdth = P.get<double>(nt);
    SB_B(P.err);
    k_triplets<true><<<grid_of(nh), kB, 0, s>>>(H, p, doff, d_out, d_theta, toff, nullptr, ta, tb,
                                                tc, tk, tdth);
    SB_B(cudaGetLastError());
    // 3. hit -> triplet incidence (ascending triplet order per hit)
    unsigned long long* hcnt = P.get<unsigned long long>(nh + 1);
    unsigned long long* hfill = P.get<unsigned long long>(nh + 1);
    long long* hoff = P.get<long long>(nh + 1);
    int32_t* list = P.get<int32_t>(3 * nt);
    SB_B(P.err);
    SB_B(cudaMemsetAsync(hcnt, 0, (nh + 1) * 8, s));
    SB_B(cudaMemsetAsync(hfill, 0, (nh + 1) * 8, s));
    k_incidence_count<<<grid_of(nt), kB, 0, s>>>(ta, tb, tc, nt, hcnt);
    SB_B(cudaGetLastError());
    long long ninc = 0;
    SB_B(exclusive_scan(reinterpret_cast<long long*>(hcnt), hoff, nh + 1, &ninc, s));
    k_incidence_fill<<<grid_of(nt), kB, 0, s>>>(ta, tb, tc, nt, hoff, hfill, list);
    SB_B(cudaGetLastError());
    k_incidence_sort<<<grid_of(nh), kB, 0, s>>>(hoff, nh, list);
    SB_B(cudaGetLastError());
    // 4. pairs
    Trip T;
    T.a = ta;
    T.b = tb;
    T.c = tc;
    T.k = tk;
    T.dth = tdth;
    T.n = nt;
    long long* pcnt = P.get<long long>(nt + 1);
    long long* poff = P.get<long long>(nt + 1);
    SB_B(P.err);
    SB_B(cudaMemsetAsync(pcnt, 0, (nt + 1) * 8, s));
    k_pairs<<<grid_of(nt), kB, 0, s>>>(H, p, T, hoff, list, nullptr, pcnt, nullptr, nullptr);
    SB_B(cudaGetLastError());
    long long np = 0;
    SB_B(exclusive_scan(pcnt, poff, nt + 1, &np, s));
    int32_t* pj = P.get<int32_t>(np);
    int8_t* pcls = P.get<int8_t>(np);
    SB_B(P.err);
    k_pairs<<<grid_of(nt), kB, 0, s>>>(H, p, T, hoff, list, poff, nullptr, pj, pcls);
    SB_B(cudaGetLastError());
    // 5. pruning
    uint8_t* has_succ = P.get<uint8_t>(nt);
    uint8_t* has_pred = P.get<uint8_t>(nt);
    uint8_t* keep = P.get<uint8_t>(nt);
    long long* keep_ll = P.get<long long>(nt + 1);
    long long* newidx = P.get<long long>(nt + 1);
    SB_B(P.err);
    SB_B(cudaMemsetAsync(has_succ, 0, std::max<long long>(nt, 1), s));
    SB_B(cudaMemsetAsync(has_pred, 0, std::max<long long>(nt, 1), s));
    SB_B(cudaMemsetAsync(keep, 0, std::max<long long>(nt, 1), s));
    SB_B(cudaMemsetAsync(keep_ll, 0, (nt + 1) * 8, s));
    k_links<<<grid_of(nt), kB, 0, s>>>(H, T, poff, pj, pcls, has_succ, has_pred);
    SB_B(cudaGetLastError());
    k_keep<<<grid_of(nt), kB, 0, s>>>(H, p, T, poff, pj, pcls, has_succ, has_pred, keep);
    SB_B(cudaGetLastError());
    k_u8_to_ll<<<grid_of(nt), kB, 0, s>>>(keep, keep_ll, nt);
    SB_B(cudaGetLastError());
    long long n = 0;
    SB_B(exclusive_scan(keep_ll, newidx, nt + 1, &n, s));
    // 6. CSR over the survivors
    long long* rcnt = P.get<long long>(n + 1);
    long long* roff = P.get<long long>(n + 1);
    SB_B(P.err);
    SB_B(cudaMemsetAsync(rcnt, 0, (n + 1) * 8, s));
    k_rows<<<grid_of(nt), kB, 0, s>>>(T, poff, pj, keep, newidx, rcnt);
    SB_B(cudaGetLastError());
    long long nnz = 0;
    SB_B(exclusive_scan(rcnt, roff, n + 1, &nnz, s));
    if (nnz >= 0x7FFFFFFFLL) return fail(cudaErrorInvalidValue);
    int32_t* col = P.get<int32_t>(nnz);
    double* val = P.get<double>(nnz);
    int8_t* cls = P.get<int8_t>(nnz);
    double* quality = P.get<double>(n);
    double* lin = P.get<double>(n);
    int32_t* trip = P.get<int32_t>(3 * n);
    double* kappa = P.get<double>(n);
    double* dtheta = P.get<double>(n);
    SB_B(P.err);
    k_rows_write<<<grid_of(nt), kB, 0, s>>>(H, p, T, poff, pj, pcls, keep, newidx, roff, col, val,
                                            cls, quality, lin, trip, kappa, dtheta);
    SB_B(cudaGetLastError());
    SB_B(cudaEventRecord(e1, s));
    // copy out
    sb_qubo* q = new (std::nothrow) sb_qubo;
    if (!q) return fail(cudaErrorMemoryAllocation);
    q->n = (int32_t)n;
    q->w_c = bp->w_c;
    q->n_hits = (int32_t)ev->layer.size();
    q->rowptr.resize(n + 1);
    q->col.resize(nnz);
    q->val.resize(nnz);
    q->cls.resize(nnz);
    q->quality.resize(n);
    q->lin.resize(n);
    q->trip.resize(3 * n);
    q->kappa.resize(n);
    q->dtheta.resize(n);
    std::vector<long long> ro(n + 1);
    cudaError_t e = cudaMemcpyAsync(ro.data(), roff, (n + 1) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nnz) {
      e = cudaMemcpyAsync(q->col.data(), col, nnz * 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(q->val.data(), val, nnz * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(q->cls.data(), cls, nnz, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess && n) {
      e = cudaMemcpyAsync(q->quality.data(), quality, n * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(q->lin.data(), lin, n * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(q->trip.data(), trip, 3 * n * 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(q->kappa.data(), kappa, n * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(q->dtheta.data(), dtheta, n * 8, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      delete q;
      return fail(e);
    }
    ro[n] = nnz;
    for (long long i = 0; i <= n; ++i) q->rowptr[i] = (int32_t)ro[i];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (out_device_ms) *out_device_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = q;
    return SB_OK;
#undef SB_B
  });
}
