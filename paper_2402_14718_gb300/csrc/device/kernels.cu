// Device kernels of the SB solver (sm_103a).
//
//  * k_convert / k_event_stats -- QUBO (Eq. 13) -> Ising in FP64.
//  * k_init                    -- Philox4x32-10 initial state.
//  * k_step                    -- one fused SB step: CSR coupling product over
//                                 the replicas (Eq. 2 / 6 / 10), symplectic-Euler
//                                 momentum and position update, inelastic wall.
//  * k_energy_partial / k_energy_reduce / k_argmin / k_best_T -- FP64 QUBO
//                                 energy of sgn(x), arg-min over replicas.
//
// State is replica-minor (element (i, r) at i * R + r): the R replicas of one
// row are contiguous, so one group of threads reading row j of X for all its
// replicas issues fully coalesced 16-byte loads.
#include <cuda_bf16.h>
#include <float.h>
#include <limits.h>

#include <algorithm>

#include "../philox.h"
#include "kernels.cuh"
#include "signs.cuh"

namespace sbd {

Tiling make_tiling(int R) {
  Tiling t;
  t.V = (R % 4 == 0) ? 4 : 1;
  t.C = R / t.V;
  int G = 1;
  while (G * 2 <= t.C && G < 32) G *= 2;
  t.G = G;
  const int per = (t.C + G - 1) / G;
  t.NCH = per <= 1 ? 1 : (per <= 2 ? 2 : 4);
  t.tiles = (t.C + G * t.NCH - 1) / (G * t.NCH);
  return t;
}

bool dsb16_ok(int R) {
  if (R % 16 != 0) return false;
  const int G = R / 16;
  return G >= 1 && G <= 32 && (G & (G - 1)) == 0;
}

Tiling make_tiling_dsb16(int R) {
  Tiling t;
  t.V = 16;
  t.G = R / 16;
  t.C = 1;
  t.NCH = 1;
  t.tiles = 1;
  return t;
}

Tiling make_tiling_rt(int R, int RT) {
  Tiling t;
  t.V = 4;
  t.C = R / 4;
  t.G = RT / 4;
  t.NCH = 1;
  t.tiles = R / RT;
  return t;
}

namespace {

constexpr int kBlock = 256;

template <int V>
struct Vec;
template <>
struct Vec<4> {
  float v[4];
  __device__ __forceinline__ void ldg(const float* p) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
  __device__ __forceinline__ void ld(const float* p) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
  __device__ __forceinline__ void st(float* p) const {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec<1> {
  float v[1];
  __device__ __forceinline__ void ldg(const float* p) { v[0] = __ldg(p); }
  __device__ __forceinline__ void ld(const float* p) { v[0] = *p; }
  __device__ __forceinline__ void st(float* p) const { *p = v[0]; }
};

// V sign bytes of one chunk as the floats 2^-7 sgn
template <int V>
__device__ __forceinline__ void ld_signs(const uint8_t* p, float (&out)[V]) {
  if (V == 4) {
    const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(p));
#pragma unroll
    for (int v = 0; v < V; ++v) out[v] = scaled_sign_of_byte(w, v);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) out[v] = scaled_sign_of_byte(__ldg(p + v), 0);
  }
}

__device__ __forceinline__ float jval(const float* J, int p) { return __ldg(J + p); }
__device__ __forceinline__ float jval(const __nv_bfloat16* J, int p) {
  return __bfloat162float(J[p]);
}


// lanes of this thread's row group inside its warp
__device__ __forceinline__ unsigned group_mask(int G) {
  const int lane = threadIdx.x & 31;
  return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// ---------------------------------------------------------------- SB step
// One row per group of G threads; the group loads G (col, J) pairs of the row
// at a time (coalesced) and broadcasts them with shuffles; every thread then
// gathers its replica chunks of the neighbour rows with 16-byte loads, four
// neighbours in flight at once.
// MODE: 0 aSB, 1 bSB, 2 dSB gathering x (sgn at use), 3 dSB gathering int8
// signs, 4 bSB also recording the pre-wall momentum and the wall mask.
// CTAs per SM the compiler is asked to fit: with two or four chunks per thread
// the free choice takes 101 / 168 registers (two / one CTA per SM); bounding it
// gives 80 / 128 registers and three / two CTAs without spills
template <int NCH>
struct StepMinBlocks {
  static constexpr int value = NCH == 2 ? 3 : (NCH == 4 ? 2 : 1);
};
template <int V, int NCH, int MODE, typename JT>
__global__ void __launch_bounds__(kBlock, StepMinBlocks<NCH>::value) k_step(const StepArgs a) {
  constexpr int VARIANT = MODE == 3 ? 2 : (MODE == 4 ? 1 : MODE);
  constexpr bool use_sgn = MODE == 3;
  constexpr bool record = MODE == 4;
  constexpr int U = 4;
  const int G = a.G;
  const int gid = threadIdx.x / G;
  const int g = threadIdx.x - gid * G;
  const int groups = blockDim.x / G;
  const unsigned mask = group_mask(G);
  const int R = a.R;
  const int C = R / V;
  const int ch0 = (blockIdx.y + a.tile0) * (G * NCH) + g;
  const JT* J = static_cast<const JT*>(a.J);
  const int row_end = min(a.n, (blockIdx.x + 1) * a.rpc);
  // a CTA walks a contiguous chunk of rows, so rows in flight together share
  // neighbour rows in L1; the group count is uniform, so a group leaves whole
  for (int row = blockIdx.x * a.rpc + gid; row < row_end; row += groups) {
  float acc[NCH][V];
#pragma unroll
  for (int j = 0; j < NCH; ++j)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[j][v] = 0.f;

  int p0 = __ldg(a.rowptr + row), p1 = __ldg(a.rowptr + row + 1);
  chk_rows(p0, p1, a.nnz);
  for (int pb = p0; pb < p1; pb += G) {
    const int cnt = min(G, p1 - pb);
    int mc = 0;
    float mv = 0.f;
    if (g < cnt) {
      mc = chk_idx(__ldg(a.col + pb + g), a.n, kChkCol);
      mv = jval(J, pb + g);
      if (use_sgn) mv *= kSignScale;  // 2^7 J: sign bytes read as 2^-7 sgn
    }
    int q = 0;
    for (; q + U <= cnt; q += U) {
      int c[U];
      float w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        c[u] = __shfl_sync(mask, mc, q + u, G);
        w[u] = __shfl_sync(mask, mv, q + u, G);
      }
      float xv[U][NCH][V];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          const int ch = ch0 + j * G;
          if (ch < C) {
            const size_t off = (size_t)c[u] * R + (size_t)ch * V;
            if (use_sgn) {
              ld_signs<V>(a.sgn_in + off, xv[u][j]);
            } else {
              Vec<V> t;
              t.ldg(a.xin + off);
#pragma unroll
              for (int v = 0; v < V; ++v) xv[u][j][v] = VARIANT == 2 ? sgnf(t.v[v]) : t.v[v];
            }
          }
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < NCH; ++j)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[j][v] = fmaf(w[u], xv[u][j][v], acc[j][v]);
    }
    for (; q < cnt; ++q) {
      const int c = __shfl_sync(mask, mc, q, G);
      const float w = __shfl_sync(mask, mv, q, G);
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int ch = ch0 + j * G;
        if (ch < C) {
          const size_t off = (size_t)c * R + (size_t)ch * V;
          float xs[V];
          if (use_sgn) {
            ld_signs<V>(a.sgn_in + off, xs);
          } else {
            Vec<V> t;
            t.ldg(a.xin + off);
#pragma unroll
            for (int v = 0; v < V; ++v) xs[v] = VARIANT == 2 ? sgnf(t.v[v]) : t.v[v];
          }
#pragma unroll
          for (int v = 0; v < V; ++v) acc[j][v] = fmaf(w, xs[v], acc[j][v]);
        }
      }
    }
  }

  // symplectic Euler: momentum with the old position, then position, then wall
  const float pa = a.a0 - __ldg(a.sched + a.k);
  const int e = a.row_event ? __ldg(a.row_event + row) : 0;
  const float c0 = __ldg(a.c0_ev + e);
  const float hi = __ldg(a.h + row);
#pragma unroll
  for (int j = 0; j < NCH; ++j) {
    const int ch = ch0 + j * G;
    if (ch >= C) continue;
    const size_t idx = (size_t)row * R + (size_t)ch * V;
    Vec<V> xv, yv;
    xv.ldg(a.xin + idx);
    yv.ld(a.y + idx);
    uint32_t sw = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float x = xv.v[v], y = yv.v[v];
      float force = -pa * x + c0 * (acc[j][v] + hi);
      if (VARIANT == 0) force -= x * x * x;
      y = y + a.dt * force;
      x = x + a.dta0 * y;
      if (record) {
        a.ytil[idx + v] = y;
        a.frec[idx + v] = acc[j][v];
      }
      const bool wall = VARIANT != 0 && fabsf(x) > 1.f;
      if (record) a.mask[idx + v] = wall ? 1 : 0;
      if (wall) {
        x = copysignf(1.f, x);
        y = 0.f;
      }
      xv.v[v] = x;
      yv.v[v] = y;
      if (VARIANT == 2) sw |= sign_byte(x) << (8 * v);
    }
    xv.st(a.xout + idx);
    yv.st(a.y + idx);
    if (use_sgn) {
      if (V == 4) {
        *reinterpret_cast<uint32_t*>(a.sgn_out + idx) = sw;
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) a.sgn_out[idx + v] = (uint8_t)((sw >> (8 * v)) & 0xff);
      }
    }
  }
  }
}

template <int V, int NCH, int MODE>
cudaError_t launch_step_t(int jbf16, const Tiling& t, const StepArgs& a, cudaStream_t s) {
  dim3 grid((a.n + a.rpc - 1) / a.rpc, t.tiles);
  if (jbf16)
    k_step<V, NCH, MODE, __nv_bfloat16><<<grid, kBlock, 0, s>>>(a);
  else
    k_step<V, NCH, MODE, float><<<grid, kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <int V, int NCH, int MODE>
int blocks_per_sm_t(int jbf16) {
  int b = 0;
  const cudaError_t e =
      jbf16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step<V, NCH, MODE, __nv_bfloat16>,
                                                            kBlock, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step<V, NCH, MODE, float>,
                                                            kBlock, 0);
  return e == cudaSuccess && b > 0 ? b : 1;
}

template <int V, int NCH>
int blocks_per_sm_v(int variant, int jbf16, int) {
  switch (variant) {
    case 0: return blocks_per_sm_t<V, NCH, 0>(jbf16);
    case 1: return blocks_per_sm_t<V, NCH, 1>(jbf16);
    default: return blocks_per_sm_t<V, NCH, 3>(jbf16);
  }
}

template <int V, int NCH>
cudaError_t launch_step_v(int variant, int jbf16, const Tiling& t, const StepArgs& a,
                          cudaStream_t s) {
  if (variant == 1 && a.ytil) return launch_step_t<V, NCH, 4>(jbf16, t, a, s);
  switch (variant) {
    case 0: return launch_step_t<V, NCH, 0>(jbf16, t, a, s);
    case 1: return launch_step_t<V, NCH, 1>(jbf16, t, a, s);
    default:
      return a.sgn_in ? launch_step_t<V, NCH, 3>(jbf16, t, a, s)
                      : launch_step_t<V, NCH, 2>(jbf16, t, a, s);
  }
}

// ---------------------------------------------------------------- one replica
// R = 1: one thread per row; eight (col, J) pairs and eight neighbour values
// are loaded before the FMAs, so a row's gathers overlap instead of forming a
// chain of dependent L2 round trips. Same CSR-order FMA sequence as k_step.
template <int MODE, typename JT>
__global__ void __launch_bounds__(kBlock) k_step_r1(const StepArgs a) {
  constexpr int VARIANT = MODE == 4 ? 1 : MODE;
  constexpr bool record = MODE == 4;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= a.n) return;
  const JT* J = static_cast<const JT*>(a.J);
  int p0 = __ldg(a.rowptr + row), p1 = __ldg(a.rowptr + row + 1);
  chk_rows(p0, p1, a.nnz);
  float acc = 0.f;
  int p = p0;
  for (; p + 8 <= p1; p += 8) {
    int c[8];
    float w[8], xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      c[u] = chk_idx(__ldg(a.col + p + u), a.n, kChkCol);
      w[u] = jval(J, p + u);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) xv[u] = __ldg(a.xin + c[u]);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = fmaf(w[u], VARIANT == 2 ? sgnf(xv[u]) : xv[u], acc);
  }
  for (; p < p1; ++p) {
    const float xv = __ldg(a.xin + chk_idx(__ldg(a.col + p), a.n, kChkCol));
    acc = fmaf(jval(J, p), VARIANT == 2 ? sgnf(xv) : xv, acc);
  }
  const float pa = a.a0 - __ldg(a.sched + a.k);
  const int e = a.row_event ? __ldg(a.row_event + row) : 0;
  const float c0 = __ldg(a.c0_ev + e);
  float x = __ldg(a.xin + row), y = a.y[row];
  float force = -pa * x + c0 * (acc + __ldg(a.h + row));
  if (VARIANT == 0) force -= x * x * x;
  y = y + a.dt * force;
  x = x + a.dta0 * y;
  if (record) {
    a.ytil[row] = y;
    a.frec[row] = acc;
  }
  const bool wall = VARIANT != 0 && fabsf(x) > 1.f;
  if (record) a.mask[row] = wall ? 1 : 0;
  if (wall) {
    x = copysignf(1.f, x);
    y = 0.f;
  }
  a.xout[row] = x;
  a.y[row] = y;
}

// One replica, G lanes per row: the lanes load the row's (col, J) and gather
// the neighbours' positions G x 4 at a time (all in flight together), then every
// lane runs the same FMA chain in CSR order over the shuffled values, so the
// sum is the one k_step_r1 forms, bit for bit, with one round trip per 4G
// neighbours instead of one per eight. Lane 0 of the group writes the row.
template <int G, int MODE, typename JT>
__global__ void __launch_bounds__(kBlock) k_step_r1g(const StepArgs a) {
  constexpr int VARIANT = MODE == 4 ? 1 : MODE;
  constexpr bool record = MODE == 4;
  constexpr int U = 4;
  const int gid = threadIdx.x / G, g = threadIdx.x - gid * G;
  const int row = blockIdx.x * (kBlock / G) + gid;
  if (row >= a.n) return;  // the whole group leaves together
  const unsigned mask = group_mask(G);
  const JT* J = static_cast<const JT*>(a.J);
  int p0 = __ldg(a.rowptr + row), p1 = __ldg(a.rowptr + row + 1);
  chk_rows(p0, p1, a.nnz);
  float acc = 0.f;
  for (int pb = p0; pb < p1; pb += G * U) {
    float w[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = pb + u * G + g;
      int c = row;
      w[u] = 0.f;
      if (p < p1) {
        c = chk_idx(__ldg(a.col + p), a.n, kChkCol);
        w[u] = jval(J, p);
      }
      xv[u] = __ldg(a.xin + c);
    }
    const int cnt = min(G * U, p1 - pb);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float s = VARIANT == 2 ? sgnf(xv[u]) : xv[u];
      const int lim = min(G, cnt - u * G);
      for (int j = 0; j < lim; ++j)
        acc = fmaf(__shfl_sync(mask, w[u], j, G), __shfl_sync(mask, s, j, G), acc);
    }
  }
  if (g != 0) return;
  const float pa = a.a0 - __ldg(a.sched + a.k);
  const int e = a.row_event ? __ldg(a.row_event + row) : 0;
  const float c0 = __ldg(a.c0_ev + e);
  float x = __ldg(a.xin + row), y = a.y[row];
  float force = -pa * x + c0 * (acc + __ldg(a.h + row));
  if (VARIANT == 0) force -= x * x * x;
  y = y + a.dt * force;
  x = x + a.dta0 * y;
  if (record) {
    a.ytil[row] = y;
    a.frec[row] = acc;
  }
  const bool wall = VARIANT != 0 && fabsf(x) > 1.f;
  if (record) a.mask[row] = wall ? 1 : 0;
  if (wall) {
    x = copysignf(1.f, x);
    y = 0.f;
  }
  a.xout[row] = x;
  a.y[row] = y;
}

// ---------------------------------------------------------------- dSB, 16 signs per lane
// dSB gathering int8 signs with 16 replicas per lane: one 16-byte load brings a
// neighbour's signs for 16 replicas. G = R / 16 lanes own a row (R / 16 a power
// of two, <= 32). Same CSR-order FMA sequence per replica as k_step.

#ifndef SB_DSB_BLOCK
#define SB_DSB_BLOCK 128
#endif
// nine CTAs of 128 threads per SM: 56 registers, no spills (measured faster
// than the unbounded 72 registers, seven CTAs; ten CTAs spill)
#ifndef SB_DSB_MINB
#define SB_DSB_MINB 9
#endif
constexpr int kDsbBlock = SB_DSB_BLOCK;  // threads per CTA of k_step_dsb16

template <typename JT>
__global__ void __launch_bounds__(kDsbBlock, SB_DSB_MINB) k_step_dsb16(const StepArgs a) {
  const int G = a.G;
  const int gid = threadIdx.x / G;
  const int g = threadIdx.x - gid * G;
  const int groups = blockDim.x / G;
  const unsigned mask = group_mask(G);
  const int R = a.R;
  const JT* J = static_cast<const JT*>(a.J);
  const int chunk = a.cta_order ? __ldg(a.cta_order + blockIdx.x) : (int)blockIdx.x;
  const int row_end = min(a.n, (chunk + 1) * a.rpc);
  for (int row = chunk * a.rpc + gid; row < row_end; row += groups) {
    float acc[16];
#pragma unroll
    for (int v = 0; v < 16; ++v) acc[v] = 0.f;
    int p0 = __ldg(a.rowptr + row), p1 = __ldg(a.rowptr + row + 1);
    chk_rows(p0, p1, a.nnz);
    for (int pb = p0; pb < p1; pb += G) {
      const int cnt = min(G, p1 - pb);
      int mc = 0;
      float mv = 0.f;
      if (g < cnt) {
        mc = chk_idx(__ldg(a.col + pb + g), a.n, kChkCol);
        mv = jval(J, pb + g);
        mv *= kSignScale;  // 2^7 J: sign bytes read as 2^-7 sgn
      }
      int q = 0;
      for (; q + 4 <= cnt; q += 4) {
        int c[4];
        float w[4];
        uint4 sv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          c[u] = __shfl_sync(mask, mc, q + u, G);
          w[u] = __shfl_sync(mask, mv, q + u, G);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          sv[u] = __ldg(reinterpret_cast<const uint4*>(a.sgn_in + (size_t)c[u] * R + 16 * g));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned ww[4] = {sv[u].x, sv[u].y, sv[u].z, sv[u].w};
#pragma unroll
          for (int v = 0; v < 16; ++v)
            acc[v] = fmaf(w[u], scaled_sign_of_byte(ww[v >> 2], v & 3), acc[v]);
        }
      }
      for (; q < cnt; ++q) {
        const int c = __shfl_sync(mask, mc, q, G);
        const float w = __shfl_sync(mask, mv, q, G);
        const uint4 s4 = __ldg(reinterpret_cast<const uint4*>(a.sgn_in + (size_t)c * R + 16 * g));
        const unsigned ww[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
        for (int v = 0; v < 16; ++v) acc[v] = fmaf(w, scaled_sign_of_byte(ww[v >> 2], v & 3), acc[v]);
      }
    }
    const float pa = a.a0 - __ldg(a.sched + a.k);
    const int e = a.row_event ? __ldg(a.row_event + row) : 0;
    const float c0 = __ldg(a.c0_ev + e);
    const float hi = __ldg(a.h + row);
    const size_t idx = (size_t)row * R + 16 * g;
    unsigned sw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int h4 = 0; h4 < 4; ++h4) {
      Vec<4> xv, yv;
      xv.ldg(a.xin + idx + 4 * h4);
      yv.ld(a.y + idx + 4 * h4);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float x = xv.v[v], y = yv.v[v];
        const float force = -pa * x + c0 * (acc[4 * h4 + v] + hi);
        y = y + a.dt * force;
        x = x + a.dta0 * y;
        if (fabsf(x) > 1.f) {
          x = copysignf(1.f, x);
          y = 0.f;
        }
        xv.v[v] = x;
        yv.v[v] = y;
        sw[h4] |= sign_byte(x) << (8 * v);
      }
      xv.st(a.xout + idx + 4 * h4);
      yv.st(a.y + idx + 4 * h4);
    }
    *reinterpret_cast<uint4*>(a.sgn_out + idx) = make_uint4(sw[0], sw[1], sw[2], sw[3]);
  }
}

// ---------------------------------------------------------------- tiled SB step
// Packed per-nonzero word of the tiled kernel: the neighbour's local index in
// the block's union and J. BF16 J: u32 = (index << 16) | bf16 bits (a BF16 value
// widens to FP32 by a 16-bit shift). FP32 J: u64 = (index, f32 bits).
template <typename JT>
struct TzWord;
template <>
struct TzWord<__nv_bfloat16> {
  typedef uint32_t T;
  static __device__ __forceinline__ int idx(uint32_t w) { return (int)(w >> 16); }
  static __device__ __forceinline__ float val(uint32_t w) { return __uint_as_float(w << 16); }
};
template <>
struct TzWord<float> {
  typedef uint2 T;
  static __device__ __forceinline__ int idx(uint2 w) { return (int)w.x; }
  static __device__ __forceinline__ float val(uint2 w) { return __uint_as_float(w.y); }
};

__device__ __forceinline__ void cp_async16(void* smem_ptr, const void* gptr) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_ptr);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gptr));
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem_ptr, const void* gptr) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_ptr);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gptr), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {  // all groups but the newest done
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

constexpr int kTiledThreads = 512;

template <typename W>
struct TiledStage {
  static constexpr size_t kX = (size_t)kTileUCap * kTileRT * sizeof(float);
  static constexpr size_t kBytes = kX + (size_t)kTileNzCap * sizeof(W);
};

// Issue the asynchronous copies of one (row block, replica tile) item into a
// pipeline stage: the union rows of x (32 replicas = 128 bytes each) and the
// block's packed (index, J) words. Row ids are read before any copy is issued.
template <typename W>
__device__ __forceinline__ void tiled_issue(const TiledArgs& a, long long item, int ntiles,
                                            unsigned char* stage) {
  const int b = (int)(item / ntiles);
  const int r_base = (int)(item - (long long)b * ntiles) * kTileRT;
  const int u0 = a.blk_u0[b], nu8 = (a.blk_u0[b + 1] - u0) * 8;
  const int row0 = a.blk_row0[b];
  const int z0 = a.rowptr[row0], nz = a.rowptr[a.blk_row0[b + 1]] - z0;
  float4* Xs = reinterpret_cast<float4*>(stage);
  W* Zs = reinterpret_cast<W*>(stage + TiledStage<W>::kX);
  constexpr int PER = kTileUCap * 8 / kTiledThreads;
  int uc[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int k = threadIdx.x + j * kTiledThreads;
    uc[j] = k < nu8 ? __ldg(a.ucol + u0 + (k >> 3)) : 0;
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int k = threadIdx.x + j * kTiledThreads;
    if (k < nu8) cp_async16(Xs + k, a.xin + (size_t)uc[j] * a.R + r_base + 4 * (k & 7));
  }
  const W* tz = static_cast<const W*>(a.tz) + z0;
  for (int k = threadIdx.x; k < nz; k += kTiledThreads) cp_async_small<sizeof(W)>(Zs + k, tz + k);
}

// Persistent CTAs (one per SM) walk the (row block, replica tile) items with a
// two-stage cp.async pipeline: the copies of the next item are in flight while
// the current one is computed. Each item: 8 lanes own a row and 4 replicas
// (float4), so every shared-memory read of a neighbour row serves 4 FMAs and a
// warp reads 4 whole 128-byte rows at once. The FMA sequence per (row,
// replica) is the CSR order, as in k_step (dSB applies sgn at use, as k_step).
template <int VARIANT, typename JT>
__global__ void __launch_bounds__(kTiledThreads, 1) k_step_tiled(const TiledArgs a) {
  typedef typename TzWord<JT>::T W;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ntiles = a.R / kTileRT;
  const long long items = (long long)a.nb * ntiles;
  long long it = blockIdx.x;
  if (it >= items) return;
  const int R = a.R;
  const float pa = a.a0 - __ldg(a.sched + a.k);
  const int slot = threadIdx.x >> 3, q = threadIdx.x & 7;
  int stage = 0;
  tiled_issue<W>(a, it, ntiles, smem);
  cp_async_commit();
  for (; it < items; it += gridDim.x) {
    const long long nxt = it + gridDim.x;
    if (nxt < items) tiled_issue<W>(a, nxt, ntiles, smem + (stage ^ 1) * TiledStage<W>::kBytes);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();

    unsigned char* st = smem + stage * TiledStage<W>::kBytes;
    const float4* Xs = reinterpret_cast<const float4*>(st);
    const W* Zs = reinterpret_cast<const W*>(st + TiledStage<W>::kX);
    const int b = (int)(it / ntiles);
    const int r_base = (int)(it - (long long)b * ntiles) * kTileRT;
    const int row0 = a.blk_row0[b], row1 = a.blk_row0[b + 1];
    const int z0 = a.rowptr[row0];
    for (int row = row0 + slot; row < row1; row += kTiledThreads / 8) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      const int p0 = a.rowptr[row] - z0, p1 = a.rowptr[row + 1] - z0;
#pragma unroll 4
      for (int p = p0; p < p1; ++p) {
        const W w = Zs[p];
        const float j = TzWord<JT>::val(w);
        float4 xv = Xs[TzWord<JT>::idx(w) * 8 + q];
        if (VARIANT == 2) xv = make_float4(sgnf(xv.x), sgnf(xv.y), sgnf(xv.z), sgnf(xv.w));
        acc.x = fmaf(j, xv.x, acc.x);
        acc.y = fmaf(j, xv.y, acc.y);
        acc.z = fmaf(j, xv.z, acc.z);
        acc.w = fmaf(j, xv.w, acc.w);
      }
      const int e = a.row_event ? __ldg(a.row_event + row) : 0;
      const float c0 = __ldg(a.c0_ev + e);
      const float hi = __ldg(a.h + row);
      const size_t idx = (size_t)row * R + r_base + 4 * q;
      const float4 xo = Xs[(int)a.own[row] * 8 + q];
      const float4 yo = *reinterpret_cast<const float4*>(a.y + idx);
      float xs[4] = {xo.x, xo.y, xo.z, xo.w};
      float ys[4] = {yo.x, yo.y, yo.z, yo.w};
      const float fs[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        float x = xs[v], y = ys[v];
        float force = -pa * x + c0 * (fs[v] + hi);
        if (VARIANT == 0) force -= x * x * x;
        y = y + a.dt * force;
        x = x + a.dta0 * y;
        if (VARIANT != 0 && fabsf(x) > 1.f) {
          x = copysignf(1.f, x);
          y = 0.f;
        }
        xs[v] = x;
        ys[v] = y;
      }
      *reinterpret_cast<float4*>(a.xout + idx) = make_float4(xs[0], xs[1], xs[2], xs[3]);
      *reinterpret_cast<float4*>(a.y + idx) = make_float4(ys[0], ys[1], ys[2], ys[3]);
    }
    __syncthreads();  // the stage is refilled by the next iteration's issue
    stage ^= 1;
  }
}

template <int VARIANT, typename JT>
cudaError_t launch_tiled_t(const TiledArgs& a, cudaStream_t s) {
  typedef typename TzWord<JT>::T W;
  const size_t smem = 2 * TiledStage<W>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(k_step_tiled<VARIANT, JT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const long long items = (long long)a.nb * (a.R / kTileRT);
  const long long grid = std::min<long long>(items, (long long)sms);
  k_step_tiled<VARIANT, JT><<<(unsigned)grid, kTiledThreads, smem, s>>>(a);
  return cudaGetLastError();
}

__global__ void k_pack_tz_bf16(const __nv_bfloat16* J, const uint16_t* lidx, int64_t nnz,
                               uint32_t* tz) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    tz[p] = ((uint32_t)lidx[p] << 16) | (uint32_t)__bfloat16_as_ushort(J[p]);
}

__global__ void k_pack_tz_f32(const float* J, const uint16_t* lidx, int64_t nnz, uint2* tz) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    tz[p] = make_uint2((uint32_t)lidx[p], __float_as_uint(J[p]));
}


// ---------------------------------------------------------------- bSB adjoint
// FP64 block sum of up to 4 values into acc[0..n) (one atomic per block and value).
__device__ __forceinline__ void block_add(double v0, double v1, double v2, double v3,
                                          double* t0, double* t1, double* t2, double* t3) {
  __shared__ double sh[4][kBlock / 32];
  double v[4] = {v0, v1, v2, v3};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) sh[q][wid] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] += sh[q][w];
    double* tg[4] = {t0, t1, t2, t3};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (tg[q]) atomicAdd(tg[q], s[q]);
  }
}

// Sparse products of one row for this thread's replica chunks:
// sJ = sum_j J_ij u_j, and (when x given) fJ = sum_j J_ij x_j, fC = sum_{conflict j} x_j.
template <int V, int NCH, typename JT, bool TWO>
__device__ __forceinline__ void adj_row_products(const AdjArgs& a, int row, int ch0, int C,
                                                 unsigned mask, const float* u, const float* xk,
                                                 float (&sJ)[NCH][V], float (&fJ)[NCH][V],
                                                 float (&fC)[NCH][V]) {
  const int G = a.G, g = ch0 % G;
  const JT* J = static_cast<const JT*>(a.J);
#pragma unroll
  for (int j = 0; j < NCH; ++j)
#pragma unroll
    for (int v = 0; v < V; ++v) sJ[j][v] = fJ[j][v] = fC[j][v] = 0.f;
  const int p0 = a.rowptr[row], p1 = a.rowptr[row + 1];
  for (int pb = p0; pb < p1; pb += G) {
    const int cnt = min(G, p1 - pb);
    int mc = 0, mk = 0;
    float mv = 0.f;
    if (g < cnt) {
      mc = a.col[pb + g];
      mv = jval(J, pb + g);
      mk = a.cls[pb + g];
    }
    for (int q = 0; q < cnt; ++q) {
      const int c = __shfl_sync(mask, mc, q, G);
      const float w = __shfl_sync(mask, mv, q, G);
      const int kc = __shfl_sync(mask, mk, q, G);
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int ch = ch0 + j * G;
        if (ch >= C) continue;
        const size_t off = (size_t)c * a.R + (size_t)ch * V;
        Vec<V> uv;
        uv.ldg(u + off);
#pragma unroll
        for (int v = 0; v < V; ++v) sJ[j][v] = fmaf(w, uv.v[v], sJ[j][v]);
        if (TWO) {
          Vec<V> xv;
          xv.ldg(xk + off);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            fJ[j][v] = fmaf(w, xv.v[v], fJ[j][v]);
            if (kc) fC[j][v] += xv.v[v];
          }
        }
      }
    }
  }
}

// lambda_x = (-J x_S - h) / R, lambda_y = 0; loss, dL/dh_i = -sum_r x_S / R and the
// explicit w_c term sum x (C x) / (8 R).
template <int V, int NCH, typename JT>
__global__ void __launch_bounds__(kBlock) k_adj_init(const AdjArgs a) {
  const int G = a.G;
  const int gid = threadIdx.x / G, g = threadIdx.x - gid * G;
  const int row = blockIdx.x * (blockDim.x / G) + gid;
  const int C = a.R / V;
  const int ch0 = blockIdx.y * (G * NCH) + g;
  double loss = 0.0, wc = 0.0, ghr = 0.0;
  if (row < a.n) {
    const unsigned mask = group_mask(G);
    float sJ[NCH][V], fJ[NCH][V], fC[NCH][V];
    adj_row_products<V, NCH, JT, true>(a, row, ch0, C, mask, a.x, a.x, sJ, fJ, fC);
    const float hi = a.h[row];
    const double invR = 1.0 / a.R;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int ch = ch0 + j * G;
      if (ch >= C) continue;
      const size_t idx = (size_t)row * a.R + (size_t)ch * V;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const double x = a.x[idx + v];
        a.lx[idx + v] = (float)((-(double)fJ[j][v] - hi) * invR);
        a.ly[idx + v] = 0.f;
        loss += (-0.5 * x * fJ[j][v] - hi * x) * invR;
        wc += x * fC[j][v] * invR / 8.0;
        ghr -= x * invR;
      }
    }
    for (int off = G / 2; off > 0; off >>= 1) ghr += __shfl_down_sync(mask, ghr, off, G);
    if (g == 0) atomicAdd(a.gh + row, ghr);
  }
  block_add(loss, wc, 0.0, 0.0, a.acc + 0, a.acc + 3, nullptr, nullptr);
}

// Through the wall: lx~ = (1 - m) lx; ly~ = (1 - m) ly + dt a0 lx~.
__global__ void k_adj_phase1(const AdjArgs a) {
  const size_t total = (size_t)a.n * a.R;
  const float dta0 = a.dt * a.a0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const bool keep = a.mask[i] == 0;
    const float lxt = keep ? a.lx[i] : 0.f;
    a.lx[i] = lxt;
    a.lyt[i] = (keep ? a.ly[i] : 0.f) + dta0 * lxt;
  }
}

// Momentum update reversed: lx_k = lx~ - dt (a0 - a_k) ly~ + dt c0 J ly~, ly_k = ly~,
// and the gradient contributions of this step. One gather of ly~ gives both
// J ly~ and C ly~ (conflict entries only); J x_k comes recorded from the
// forward recomputation, and sum ly~ (C x_k) = sum x_k (C ly~) since C is
// symmetric. Each element's gradient terms are products of FP32 values formed
// in FP32 and summed in FP64 (FP64 arithmetic is scarce on this part). A
// block walks several row groups (grid-stride), so only a few blocks per SM
// add their sums into the shared FP64 totals.
template <int V, int NCH, typename JT>
__global__ void __launch_bounds__(kBlock) k_adj_phase2(const AdjArgs a) {
  const int G = a.G;
  const int gid = threadIdx.x / G, g = threadIdx.x - gid * G;
  const int C = a.R / V;
  const int ch0 = blockIdx.y * (G * NCH) + g;
  double gdt = 0.0, gc0 = 0.0, ga = 0.0, gwc = 0.0;
  const int rstep = gridDim.x * (blockDim.x / G);
  for (int row = blockIdx.x * (blockDim.x / G) + gid; row < a.n; row += rstep) {
    double ghr = 0.0;
    const unsigned mask = group_mask(G);
    const JT* J = static_cast<const JT*>(a.J);
    float sJ[NCH][V], sC[NCH][V];
#pragma unroll
    for (int j = 0; j < NCH; ++j)
#pragma unroll
      for (int v = 0; v < V; ++v) sJ[j][v] = sC[j][v] = 0.f;
    const int p0 = a.rowptr[row], p1 = a.rowptr[row + 1];
    for (int pb = p0; pb < p1; pb += G) {
      const int cnt = min(G, p1 - pb);
      int mc = 0, mk = 0;
      float mv = 0.f;
      if (g < cnt) {
        mc = a.col[pb + g];
        mv = jval(J, pb + g);
        mk = a.cls[pb + g];
      }
      int q = 0;
      for (; q + 4 <= cnt; q += 4) {  // four neighbours' loads in flight, then their FMAs in order
        int c[4], kc[4];
        float w[4];
        Vec<V> uv[4][NCH];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          c[u] = __shfl_sync(mask, mc, q + u, G);
          w[u] = __shfl_sync(mask, mv, q + u, G);
          kc[u] = __shfl_sync(mask, mk, q + u, G);
#pragma unroll
          for (int j = 0; j < NCH; ++j) {
            const int ch = ch0 + j * G;
            if (ch < C) uv[u][j].ldg(a.lyt + (size_t)c[u] * a.R + (size_t)ch * V);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int j = 0; j < NCH; ++j) {
            const int ch = ch0 + j * G;
            if (ch >= C) continue;
#pragma unroll
            for (int v = 0; v < V; ++v) {
              sJ[j][v] = fmaf(w[u], uv[u][j].v[v], sJ[j][v]);
              if (kc[u]) sC[j][v] += uv[u][j].v[v];
            }
          }
      }
      for (; q < cnt; ++q) {
        const int c = __shfl_sync(mask, mc, q, G);
        const float w = __shfl_sync(mask, mv, q, G);
        const int kc = __shfl_sync(mask, mk, q, G);
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          const int ch = ch0 + j * G;
          if (ch >= C) continue;
          Vec<V> uv;
          uv.ldg(a.lyt + (size_t)c * a.R + (size_t)ch * V);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            sJ[j][v] = fmaf(w, uv.v[v], sJ[j][v]);
            if (kc) sC[j][v] += uv.v[v];
          }
        }
      }
    }
    const float hi = a.h[row];
    const float pa = a.a0 - __ldg(a.sched + a.k);
    const float dtc0 = a.dt * a.c0;
    const float dta0 = a.dt * a.a0;
    float tdt = 0.f, tc0 = 0.f, ta = 0.f, twc = 0.f, thr = 0.f;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int ch = ch0 + j * G;
      if (ch >= C) continue;
      const size_t idx = (size_t)row * a.R + (size_t)ch * V;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float x = a.x[idx + v];
        const float lyt = a.lyt[idx + v];
        const float lxt = a.lx[idx + v];
        const float fh = a.frec[idx + v] + hi;
        const float F = -pa * x + a.c0 * fh;
        tdt += lyt * F + lxt * a.a0 * a.ytil[idx + v];
        tc0 += lyt * a.dt * fh;
        ta += lyt * a.dt * x;
        twc += dtc0 * x * (-0.25f * sC[j][v]);
        thr += dtc0 * lyt;
        const float lxk = lxt - a.dt * pa * lyt + a.dt * a.c0 * sJ[j][v];
        if (a.mask_prev) {  // phase 1 of step k - 1 on this element (as k_adj_phase1)
          const bool keep = a.mask_prev[idx + v] == 0;
          const float lxp = keep ? lxk : 0.f;
          a.lx[idx + v] = lxp;
          a.lyt_out[idx + v] = (keep ? lyt : 0.f) + dta0 * lxp;
        } else {
          a.lx[idx + v] = lxk;
          a.ly[idx + v] = lyt;
        }
      }
    }
    gdt += tdt;
    gc0 += tc0;
    ga += ta;
    gwc += twc;
    ghr = thr;
    for (int off = G / 2; off > 0; off >>= 1) ghr += __shfl_down_sync(mask, ghr, off, G);
    if (g == 0) atomicAdd(a.gh + row, ghr);
  }
  block_add(gdt, gc0, gwc, ga, a.acc + 1, a.acc + 2, a.acc + 3, a.ga);
}

__global__ void k_adj_final(const AdjArgs a, double* out) {
  double wq = 0.0, wc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    wq += a.gh[i] * (-a.quality[i] / 2.0);
    wc += a.gh[i] * (-a.nconf[i] / 4.0);
  }
  block_add(wq, wc, 0.0, 0.0, out, out + 1, nullptr, nullptr);
}

template <int V, int NCH>
cudaError_t launch_adj_vn(int which, int jbf16, const Tiling& t, const AdjArgs& a,
                          cudaStream_t s) {
  const int groups = kBlock / t.G;
  dim3 grid((a.n + groups - 1) / groups, t.tiles);
  if (which == 0) {
    if (jbf16)
      k_adj_init<V, NCH, __nv_bfloat16><<<grid, kBlock, 0, s>>>(a);
    else
      k_adj_init<V, NCH, float><<<grid, kBlock, 0, s>>>(a);
  } else {
    // a few blocks per SM walk the rows, so few blocks add into the FP64 totals
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      grid.x = std::min<unsigned>(grid.x, (unsigned)std::max(1, 4 * sms / (int)grid.y));
    if (jbf16)
      k_adj_phase2<V, NCH, __nv_bfloat16><<<grid, kBlock, 0, s>>>(a);
    else
      k_adj_phase2<V, NCH, float><<<grid, kBlock, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_sparse(int which, int jbf16, const Tiling& t, const AdjArgs& a,
                              cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (t.V == 4) {
    if (t.NCH == 1) return launch_adj_vn<4, 1>(which, jbf16, t, a, s);
    if (t.NCH == 2) return launch_adj_vn<4, 2>(which, jbf16, t, a, s);
    return launch_adj_vn<4, 4>(which, jbf16, t, a, s);
  }
  if (t.NCH == 1) return launch_adj_vn<1, 1>(which, jbf16, t, a, s);
  if (t.NCH == 2) return launch_adj_vn<1, 2>(which, jbf16, t, a, s);
  return launch_adj_vn<1, 4>(which, jbf16, t, a, s);
}
// ---------------------------------------------------------------- init / schedule
__global__ void k_init(float* x, float* y, const int32_t* row_event, const int32_t* ev_row0,
                       int32_t n, int32_t R, uint32_t k0, uint32_t k1) {
  const size_t total = (size_t)n * R;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int32_t i = (int32_t)(idx / R), r = (int32_t)(idx - (size_t)i * R);
    const int32_t e = row_event ? row_event[i] : 0;
    const int32_t il = row_event ? i - ev_row0[e] : i;
    const sbk::U32x4 w =
        sbk::philox4x32_10((uint32_t)il, (uint32_t)r, sbk::kPurposeInit, (uint32_t)e, k0, k1);
    x[idx] = sbk::init_value(w.v[0]);
    y[idx] = sbk::init_value(w.v[1]);
  }
}

__global__ void k_linear_schedule(float* sched, int32_t steps, double a0) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < steps; k += gridDim.x * blockDim.x)
    sched[k] = steps > 1 ? (float)(a0 * (double)k / (double)(steps - 1)) : 0.f;
}

__global__ void k_set_c0(float* c0_ev, const double* c0_auto, double c0, int32_t E) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
    c0_ev[e] = (float)(c0 > 0.0 ? c0 : (c0 < 0.0 ? -c0 * c0_auto[e] : c0_auto[e]));
}

// ---------------------------------------------------------------- QUBO -> Ising (FP64)
__device__ __forceinline__ void store_j(float* J, int p, double v) { J[p] = (float)v; }
__device__ __forceinline__ void store_j(__nv_bfloat16* J, int p, double v) {
  J[p] = __double2bfloat16(v);
}

template <typename JT>
__global__ void k_convert(const int32_t* rowptr, const int32_t* col, const double* qval,
                          const double* qlin, int32_t n, JT* J, double* h64, float* h32,
                          double* row_off, double* row_sq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0, lo = 0.0, sq = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const double b = qval[p];
      s += b;
      const double jv = -b / 4.0;
      store_j(J, p, jv);
      sq += jv * jv;
      if (col[p] < i) lo += b;
    }
    const double hv = -(qlin[i] / 2.0 + s / 4.0);
    h64[i] = hv;
    h32[i] = (float)hv;
    row_off[i] = qlin[i] / 2.0 + lo / 4.0;
    row_sq[i] = sq;
  }
}

// one block per event: fixed-order tree reduction of the per-row terms
__global__ void k_event_stats(const double* row_off, const double* row_sq,
                              const int32_t* ev_row0, double* offset, double* sigma,
                              double* c0_auto) {
  __shared__ double so[kBlock], ss[kBlock];
  const int e = blockIdx.x;
  const int r0 = ev_row0[e], r1 = ev_row0[e + 1];
  double a = 0.0, b = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    a += row_off[i];
    b += row_sq[i];
  }
  so[threadIdx.x] = a;
  ss[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      so[threadIdx.x] += so[threadIdx.x + w];
      ss[threadIdx.x] += ss[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double n = (double)(r1 - r0);
    const double sg = n >= 2.0 ? sqrt(ss[0] / (n * (n - 1.0))) : 0.0;
    offset[e] = so[0];
    sigma[e] = sg;
    c0_auto[e] = sg > 0.0 ? 0.5 / (sqrt(n) * sg) : 1.0;
  }
}

// ---------------------------------------------------------------- FP64 energy
template <int V>
__device__ __forceinline__ void load_T(const EnergyArgs& a, size_t idx, double (&t)[V]) {
  if (a.x) {
    Vec<V> xv;
    xv.ldg(a.x + idx);
#pragma unroll
    for (int v = 0; v < V; ++v) t[v] = xv.v[v] > 0.f ? 1.0 : 0.0;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) t[v] = a.spins[idx + v] > 0 ? 1.0 : 0.0;
  }
}

// Block b sums, for every replica, T_i (a_i + 1/2 sum_j b_ij T_j) over its rows
// (Eq. 13 written with both CSR triangles), then reduces its groups in fixed order.
template <int V, int NCH>
__global__ void __launch_bounds__(kBlock) k_energy_partial(const EnergyArgs a) {
  extern __shared__ double sm[];
  const int G = a.G;
  const int gid = threadIdx.x / G;
  const int g = threadIdx.x - gid * G;
  const int groups = blockDim.x / G;
  const unsigned mask = group_mask(G);
  const int R = a.R;
  const int C = R / V;
  const int tile_base = blockIdx.y * (G * NCH);
  const int ch0 = tile_base + g;
  const int b = blockIdx.x;
  const int r0 = a.blk_row[b], r1 = a.blk_row[b + 1];
  double acc[NCH][V];
#pragma unroll
  for (int j = 0; j < NCH; ++j)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[j][v] = 0.0;
  for (int row = r0 + gid; row < r1; row += groups) {
    double inner[NCH][V];
#pragma unroll
    for (int j = 0; j < NCH; ++j)
#pragma unroll
      for (int v = 0; v < V; ++v) inner[j][v] = 0.0;
    int p0 = a.rowptr[row], p1 = a.rowptr[row + 1];
    chk_rows(p0, p1, a.nnz);
    for (int pb = p0; pb < p1; pb += G) {
      const int cnt = min(G, p1 - pb);
      int mc = 0;
      double mv = 0.0;
      if (g < cnt) {
        mc = chk_idx(a.col[pb + g], a.n, kChkCol);
        mv = a.qval[pb + g];
      }
      for (int q = 0; q < cnt; ++q) {
        const int c = __shfl_sync(mask, mc, q, G);
        const double w = __shfl_sync(mask, mv, q, G);
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          const int ch = ch0 + j * G;
          if (ch < C) {
            double t[V];
            load_T<V>(a, (size_t)c * R + (size_t)ch * V, t);
#pragma unroll
            for (int v = 0; v < V; ++v) inner[j][v] += w * t[v];
          }
        }
      }
    }
    const double ai = a.qlin[row];
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int ch = ch0 + j * G;
      if (ch < C) {
        double t[V];
        load_T<V>(a, (size_t)row * R + (size_t)ch * V, t);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[j][v] += t[v] * (ai + 0.5 * inner[j][v]);
      }
    }
  }
  const int W = G * NCH * V;
#pragma unroll
  for (int j = 0; j < NCH; ++j)
#pragma unroll
    for (int v = 0; v < V; ++v) sm[gid * W + (j * G + g) * V + v] = acc[j][v];
  __syncthreads();
  for (int t = threadIdx.x; t < W; t += blockDim.x) {
    const int rep = tile_base * V + t;
    if (rep >= R) continue;
    double s = 0.0;
    for (int k = 0; k < groups; ++k) s += sm[k * W + t];
    a.partial[(size_t)b * R + rep] = s;
  }
}

__global__ void k_energy_reduce(const double* partial, const int32_t* ev_blk0, int32_t R,
                                double* out) {
  const int e = blockIdx.y;
  const int b0 = ev_blk0[e], b1 = ev_blk0[e + 1];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = b0; b < b1; ++b) s += partial[(size_t)b * R + r];
    out[(size_t)e * R + r] = s;
  }
}

__device__ __forceinline__ bool better(double v, int r, double bv, int br) {
  return v < bv || (v == bv && r < br);
}

// warp-shuffle arg-min over the replicas of one event
__global__ void k_argmin(const double* E_all, int32_t R, double* best_E, int32_t* best_r) {
  __shared__ double sv[32];
  __shared__ int sr[32];
  const int e = blockIdx.x;
  double bv = DBL_MAX;
  int br = INT_MAX;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double v = E_all[(size_t)e * R + r];
    if (better(v, r, bv, br)) {
      bv = v;
      br = r;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, bv, off);
    const int orr = __shfl_down_sync(0xffffffffu, br, off);
    if (better(ov, orr, bv, br)) {
      bv = ov;
      br = orr;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sv[wid] = bv;
    sr[wid] = br;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    bv = lane < nw ? sv[lane] : DBL_MAX;
    br = lane < nw ? sr[lane] : INT_MAX;
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, off);
      const int orr = __shfl_down_sync(0xffffffffu, br, off);
      if (better(ov, orr, bv, br)) {
        bv = ov;
        br = orr;
      }
    }
    if (lane == 0) {
      best_E[e] = bv;
      best_r[e] = br == INT_MAX ? 0 : br;
    }
  }
}

__global__ void k_best_T(const float* x, const int32_t* row_event, const int32_t* best_r,
                         int32_t n, int32_t R, uint8_t* T) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = row_event ? row_event[i] : 0;
    T[i] = x[(size_t)i * R + best_r[e]] > 0.f ? 1 : 0;
  }
}

template <int V, int NCH>
cudaError_t launch_energy_t(const Tiling& t, const EnergyArgs& a, cudaStream_t s) {
  const int groups = kBlock / t.G;
  const size_t smem = (size_t)groups * t.G * t.NCH * t.V * sizeof(double);
  dim3 grid(a.nblk, t.tiles);
  k_energy_partial<V, NCH><<<grid, kBlock, smem, s>>>(a);
  return cudaGetLastError();
}

int grid_for(size_t work, int block) {
  size_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

}  // namespace

int dsb16_rows_per_cta(int rpc) {
  return rpc * kDsbBlock / kBlock > 0 ? rpc * kDsbBlock / kBlock : 1;
}


cudaError_t launch_step(int variant, int jbf16, const Tiling& t, const StepArgs& a,
                        cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (a.R == 1 && !a.sgn_in && a.rpc == 256 / t.G) {
    const int mode = (variant == 1 && a.ytil) ? 4 : variant;
    if (a.r1_lanes == 8 || a.r1_lanes == 16 || a.r1_lanes == 32) {
      const int grid = (int)(((int64_t)a.n * a.r1_lanes + kBlock - 1) / kBlock);
#define SB_R1G(GG, M)                                                                 \
  (jbf16 ? (k_step_r1g<GG, M, __nv_bfloat16><<<grid, kBlock, 0, s>>>(a), 0) \
         : (k_step_r1g<GG, M, float><<<grid, kBlock, 0, s>>>(a), 0))
#define SB_R1G_M(GG)                \
  switch (mode) {                   \
    case 0: SB_R1G(GG, 0); break;   \
    case 1: SB_R1G(GG, 1); break;   \
    case 2: SB_R1G(GG, 2); break;   \
    default: SB_R1G(GG, 4); break;  \
  }
      if (a.r1_lanes == 8) {
        SB_R1G_M(8)
      } else if (a.r1_lanes == 16) {
        SB_R1G_M(16)
      } else {
        SB_R1G_M(32)
      }
#undef SB_R1G_M
#undef SB_R1G
      return cudaGetLastError();
    }
    const int grid = (a.n + kBlock - 1) / kBlock;
#define SB_R1(M)                                                        \
  (jbf16 ? (k_step_r1<M, __nv_bfloat16><<<grid, kBlock, 0, s>>>(a), 0) \
         : (k_step_r1<M, float><<<grid, kBlock, 0, s>>>(a), 0))
    switch (mode) {
      case 0: SB_R1(0); break;
      case 1: SB_R1(1); break;
      case 2: SB_R1(2); break;
      default: SB_R1(4); break;
    }
#undef SB_R1
    return cudaGetLastError();
  }
  if (variant == 2 && a.sgn_in && a.G * 16 == a.R && t.tiles == 1 && t.V == 16) {
    // a CTA walks rpc rows (one row per G-lane group at 256 threads)
    const int rpc = dsb16_rows_per_cta(a.rpc);
    StepArgs b = a;
    b.rpc = rpc;
    dim3 grid((a.n + rpc - 1) / rpc, 1);
    if (jbf16)
      k_step_dsb16<__nv_bfloat16><<<grid, kDsbBlock, 0, s>>>(b);
    else
      k_step_dsb16<float><<<grid, kDsbBlock, 0, s>>>(b);
    return cudaGetLastError();
  }
  if (t.V == 16) return cudaErrorInvalidValue;  // that tiling needs the dSB sign bytes
  if (t.V == 4) {
    if (t.NCH == 1) return launch_step_v<4, 1>(variant, jbf16, t, a, s);
    if (t.NCH == 2) return launch_step_v<4, 2>(variant, jbf16, t, a, s);
    return launch_step_v<4, 4>(variant, jbf16, t, a, s);
  }
  if (t.NCH == 1) return launch_step_v<1, 1>(variant, jbf16, t, a, s);
  if (t.NCH == 2) return launch_step_v<1, 2>(variant, jbf16, t, a, s);
  return launch_step_v<1, 4>(variant, jbf16, t, a, s);
}

int step_blocks_per_sm(int variant, int jbf16, const Tiling& t, int unroll) {
  if (t.V == 4) {
    if (t.NCH == 1) return blocks_per_sm_v<4, 1>(variant, jbf16, unroll);
    if (t.NCH == 2) return blocks_per_sm_v<4, 2>(variant, jbf16, unroll);
    return blocks_per_sm_v<4, 4>(variant, jbf16, unroll);
  }
  if (t.NCH == 1) return blocks_per_sm_v<1, 1>(variant, jbf16, unroll);
  if (t.NCH == 2) return blocks_per_sm_v<1, 2>(variant, jbf16, unroll);
  return blocks_per_sm_v<1, 4>(variant, jbf16, unroll);
}

__global__ void k_signs(const float* x, uint8_t* s, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    s[i] = (uint8_t)sign_byte(x[i]);
}

cudaError_t launch_signs(const float* x, uint8_t* s, size_t count, cudaStream_t st) {
  if (!count) return cudaSuccess;
  k_signs<<<grid_for(count, kBlock), kBlock, 0, st>>>(x, s, count);
  return cudaGetLastError();
}

cudaError_t launch_step_tiled(int variant, int jbf16, const TiledArgs& a, cudaStream_t s) {
  if (a.nb <= 0) return cudaSuccess;
  switch (variant * 2 + (jbf16 ? 1 : 0)) {
    case 0: return launch_tiled_t<0, float>(a, s);
    case 1: return launch_tiled_t<0, __nv_bfloat16>(a, s);
    case 2: return launch_tiled_t<1, float>(a, s);
    case 3: return launch_tiled_t<1, __nv_bfloat16>(a, s);
    case 4: return launch_tiled_t<2, float>(a, s);
    default: return launch_tiled_t<2, __nv_bfloat16>(a, s);
  }
}

cudaError_t launch_pack_tz(const void* J, int jbf16, const uint16_t* lidx, int64_t nnz, void* tz,
                           cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  const int grid = grid_for((size_t)nnz, kBlock);
  if (jbf16)
    k_pack_tz_bf16<<<grid, kBlock, 0, s>>>(static_cast<const __nv_bfloat16*>(J), lidx, nnz,
                                           static_cast<uint32_t*>(tz));
  else
    k_pack_tz_f32<<<grid, kBlock, 0, s>>>(static_cast<const float*>(J), lidx, nnz,
                                          static_cast<uint2*>(tz));
  return cudaGetLastError();
}

cudaError_t launch_adj_init(int jbf16, const Tiling& t, const AdjArgs& a, cudaStream_t s) {
  return launch_adj_sparse(0, jbf16, t, a, s);
}

cudaError_t launch_adj_phase2(int jbf16, const Tiling& t, const AdjArgs& a, cudaStream_t s) {
  return launch_adj_sparse(1, jbf16, t, a, s);
}

cudaError_t launch_adj_phase1(const AdjArgs& a, cudaStream_t s) {
  const size_t total = (size_t)a.n * a.R;
  if (!total) return cudaSuccess;
  k_adj_phase1<<<grid_for(total, kBlock), kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adj_final(const AdjArgs& a, double* out, cudaStream_t s) {
  k_adj_final<<<grid_for(a.n, kBlock), kBlock, 0, s>>>(a, out);
  return cudaGetLastError();
}

cudaError_t launch_init(float* x, float* y, const int32_t* row_event, const int32_t* ev_row0,
                        int32_t n, int32_t R, uint64_t seed, cudaStream_t s) {
  const size_t total = (size_t)n * R;
  if (!total) return cudaSuccess;
  k_init<<<grid_for(total, kBlock), kBlock, 0, s>>>(x, y, row_event, ev_row0, n, R,
                                                     (uint32_t)(seed & 0xFFFFFFFFu),
                                                     (uint32_t)(seed >> 32));
  return cudaGetLastError();
}

cudaError_t launch_linear_schedule(float* sched, int32_t steps, double a0, cudaStream_t s) {
  if (steps <= 0) return cudaSuccess;
  k_linear_schedule<<<grid_for(steps, kBlock), kBlock, 0, s>>>(sched, steps, a0);
  return cudaGetLastError();
}

cudaError_t launch_set_c0(float* c0_ev, const double* c0_auto, double c0, int32_t E,
                          cudaStream_t s) {
  k_set_c0<<<grid_for(E, kBlock), kBlock, 0, s>>>(c0_ev, c0_auto, c0, E);
  return cudaGetLastError();
}

cudaError_t launch_convert(const int32_t* rowptr, const int32_t* col, const double* qval,
                           const double* qlin, int32_t n, void* J, int jbf16, double* h64,
                           float* h32, double* row_off, double* row_sq, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = grid_for(n, kBlock);
  if (jbf16)
    k_convert<__nv_bfloat16><<<grid, kBlock, 0, s>>>(rowptr, col, qval, qlin, n,
                                                     static_cast<__nv_bfloat16*>(J), h64, h32,
                                                     row_off, row_sq);
  else
    k_convert<float><<<grid, kBlock, 0, s>>>(rowptr, col, qval, qlin, n, static_cast<float*>(J),
                                             h64, h32, row_off, row_sq);
  return cudaGetLastError();
}

cudaError_t launch_event_stats(const double* row_off, const double* row_sq,
                               const int32_t* ev_row0, int32_t E, double* offset,
                               double* sigma, double* c0_auto, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  k_event_stats<<<E, kBlock, 0, s>>>(row_off, row_sq, ev_row0, offset, sigma, c0_auto);
  return cudaGetLastError();
}

cudaError_t launch_energy_partial(const Tiling& t, const EnergyArgs& a, cudaStream_t s) {
  if (a.nblk <= 0) return cudaSuccess;
  if (t.V == 4) {
    if (t.NCH == 1) return launch_energy_t<4, 1>(t, a, s);
    if (t.NCH == 2) return launch_energy_t<4, 2>(t, a, s);
    return launch_energy_t<4, 4>(t, a, s);
  }
  if (t.NCH == 1) return launch_energy_t<1, 1>(t, a, s);
  if (t.NCH == 2) return launch_energy_t<1, 2>(t, a, s);
  return launch_energy_t<1, 4>(t, a, s);
}

cudaError_t launch_energy_reduce(const double* partial, const int32_t* ev_blk0, int32_t E,
                                 int32_t R, double* E_out, cudaStream_t s) {
  if (E <= 0 || R <= 0) return cudaSuccess;
  dim3 grid((R + kBlock - 1) / kBlock, E);
  k_energy_reduce<<<grid, kBlock, 0, s>>>(partial, ev_blk0, R, E_out);
  return cudaGetLastError();
}

cudaError_t launch_argmin(const double* E_all, int32_t E, int32_t R, double* best_E,
                          int32_t* best_r, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  k_argmin<<<E, kBlock, 0, s>>>(E_all, R, best_E, best_r);
  return cudaGetLastError();
}

cudaError_t launch_best_T(const float* x, const int32_t* row_event, const int32_t* best_r,
                          int32_t n, int32_t R, uint8_t* T, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_best_T<<<grid_for(n, kBlock), kBlock, 0, s>>>(x, row_event, best_r, n, R, T);
  return cudaGetLastError();
}

SB_CHECK_READER(chk_read_kernels)

}  // namespace sbd
