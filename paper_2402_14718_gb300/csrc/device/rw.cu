// k_step_rw: one SB step (coupling product of Eq. 2 / 6 / 10, symplectic
// Euler update, inelastic wall) computed by row groups.
//
// A warp owns a group of RW rows (chosen on the host to share neighbours) and
// walks the sorted union of their columns.
// Each union entry carries the column, an RW-bit mask of the group rows that
// use it, and those rows' J values. The warp loads the neighbour row of x (its
// 128 * NCH replicas, 16-byte loads) once per entry and applies it to every
// group row in the mask, so x rows shared by neighbouring triplets are read
// once per group instead of once per row. The mask is the same for all lanes,
// so the per-row branches do not diverge. Each (row, replica) still takes one
// FMA per nonzero in ascending column order: the results equal k_step's bit
// for bit.
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.cuh"
#include "signs.cuh"

namespace sbd {
namespace {

// union entries in flight per warp (x rows loaded before their FMAs) and the
// launch-bounds residency hint; defaults measured best on the 1000-track event
#ifndef SB_RW_UB_NCH2
#define SB_RW_UB_NCH2 2
#endif
#ifndef SB_RW_UB_NCH1
#define SB_RW_UB_NCH1 4
#endif
#ifndef SB_RW_MINB
#define SB_RW_MINB 1
#endif

// RW J values of one entry, read by one lane and broadcast by shuffles.
template <int RW, typename JT>
struct JPack;
template <>
struct JPack<4, __nv_bfloat16> {
  uint2 v;
  __device__ __forceinline__ void ld(const void* base, int e) {
    v = __ldg(static_cast<const uint2*>(base) + e);
  }
  __device__ __forceinline__ JPack shfl(int src) const {
    JPack p;
    p.v.x = __shfl_sync(0xffffffffu, v.x, src);
    p.v.y = __shfl_sync(0xffffffffu, v.y, src);
    return p;
  }
  // BF16 -> FP32 is exact: the BF16 bits are the upper half of the FP32 word
  __device__ __forceinline__ float get(int q) const {
    const uint32_t w = q < 2 ? v.x : v.y;
    return __uint_as_float((q & 1) ? (w & 0xffff0000u) : (w << 16));
  }
  __device__ __forceinline__ void zero() { v = make_uint2(0u, 0u); }
};
template <>
struct JPack<2, __nv_bfloat16> {
  uint32_t v;
  __device__ __forceinline__ void ld(const void* base, int e) {
    v = __ldg(static_cast<const uint32_t*>(base) + e);
  }
  __device__ __forceinline__ JPack shfl(int src) const {
    JPack p;
    p.v = __shfl_sync(0xffffffffu, v, src);
    return p;
  }
  __device__ __forceinline__ float get(int q) const {
    return __uint_as_float((q & 1) ? (v & 0xffff0000u) : (v << 16));
  }
  __device__ __forceinline__ void zero() { v = 0u; }
};
template <>
struct JPack<4, float> {
  float4 v;
  __device__ __forceinline__ void ld(const void* base, int e) {
    v = __ldg(static_cast<const float4*>(base) + e);
  }
  __device__ __forceinline__ JPack shfl(int src) const {
    JPack p;
    p.v.x = __shfl_sync(0xffffffffu, v.x, src);
    p.v.y = __shfl_sync(0xffffffffu, v.y, src);
    p.v.z = __shfl_sync(0xffffffffu, v.z, src);
    p.v.w = __shfl_sync(0xffffffffu, v.w, src);
    return p;
  }
  __device__ __forceinline__ float get(int q) const {
    return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
  }
  __device__ __forceinline__ void zero() { v = make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct JPack<2, float> {
  float2 v;
  __device__ __forceinline__ void ld(const void* base, int e) {
    v = __ldg(static_cast<const float2*>(base) + e);
  }
  __device__ __forceinline__ JPack shfl(int src) const {
    JPack p;
    p.v.x = __shfl_sync(0xffffffffu, v.x, src);
    p.v.y = __shfl_sync(0xffffffffu, v.y, src);
    return p;
  }
  __device__ __forceinline__ float get(int q) const { return q == 0 ? v.x : v.y; }
  __device__ __forceinline__ void zero() { v = make_float2(0.f, 0.f); }
};


// MODE: 0 aSB, 1 bSB, 2 dSB gathering x (sgn at use), 3 dSB gathering the
// sign bytes written by the previous step (4 bytes per lane chunk)
template <int RW, int NCH, int MODE, typename JT>
__global__ void __launch_bounds__(kRwBlock, SB_RW_MINB) k_step_rw(const RwArgs a) {
  constexpr int VARIANT = MODE == 3 ? 2 : MODE;
  constexpr bool use_sgn = MODE == 3;
  using P = JPack<RW, JT>;
  constexpr int UB = NCH == 2 ? SB_RW_UB_NCH2 : SB_RW_UB_NCH1;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int R = a.R;
  const size_t rep0 = (size_t)blockIdx.y * (128 * NCH) + 4 * lane;  // this lane's first replica
  // byte address of (row 0, this lane's replicas); a neighbour row adds col * 4R bytes
  const char* xl = use_sgn ? reinterpret_cast<const char*>(a.sgn_in + rep0)
                           : reinterpret_cast<const char*>(a.xin + rep0);
  const unsigned rb = (use_sgn ? 1u : 4u) * (unsigned)R;
  const int chunk = a.cta_order ? __ldg(a.cta_order + blockIdx.x) : (int)blockIdx.x;
  const int g_end = min(a.ngroups, (chunk + 1) * a.gpc);
  const float pa = a.a0 - __ldg(a.sched + a.k);
  for (int grp = chunk * a.gpc + wid; grp < g_end; grp += kRwBlock / 32) {
    float acc[RW][NCH][4];
#pragma unroll
    for (int q = 0; q < RW; ++q)
#pragma unroll
      for (int j = 0; j < NCH; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[q][j][v] = 0.f;
    const int e0 = __ldg(a.gptr + grp), e1 = __ldg(a.gptr + grp + 1);
    // union entries 32 at a time, one per lane (lanes past the end hold column
    // 0 with an empty mask); the next 32 are loaded ahead
    int pk = 0;
    P jp;
    jp.zero();
    if (e0 + lane < e1) {
      pk = __ldg(a.ent + e0 + lane);
      jp.ld(a.ejv, e0 + lane);
    }
    for (int eb = e0; eb < e1; eb += 32) {
      const int cnt = min(32, e1 - eb);
      int pkn = 0;
      P jpn;
      jpn.zero();
      if (eb + 32 + lane < e1) {
        pkn = __ldg(a.ent + eb + 32 + lane);
        jpn.ld(a.ejv, eb + 32 + lane);
      }
      for (int q0 = 0; q0 < cnt; q0 += UB) {
        uint32_t m[UB];
        P w[UB];
        float xv[UB][NCH][4];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const unsigned v = (unsigned)__shfl_sync(0xffffffffu, pk, q0 + u);
          w[u] = jp.shfl(q0 + u);
          m[u] = v & 15u;
          const unsigned cu = (unsigned)chk_idx((int)(v >> 4), a.xrows > 0 ? a.xrows : a.n, kChkEntry);
          if (use_sgn) {
            const uint32_t* ps = reinterpret_cast<const uint32_t*>(xl + (size_t)cu * rb);
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
              const uint32_t t = __ldg(ps + 32 * j);
#pragma unroll
              for (int k = 0; k < 4; ++k) xv[u][j][k] = scaled_sign_of_byte(t, k);
            }
          } else {
            const float4* px = reinterpret_cast<const float4*>(xl + (size_t)cu * rb);
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
              const float4 t = __ldg(px + 32 * j);
              xv[u][j][0] = t.x;
              xv[u][j][1] = t.y;
              xv[u][j][2] = t.z;
              xv[u][j][3] = t.w;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          if (MODE == 2) {
#pragma unroll
            for (int j = 0; j < NCH; ++j)
#pragma unroll
              for (int v = 0; v < 4; ++v) xv[u][j][v] = sgnf(xv[u][j][v]);
          }
#pragma unroll
          for (int q = 0; q < RW; ++q)
            if (m[u] & (1u << q)) {
              float wq = w[u].get(q);
              if (use_sgn) wq *= kSignScale;  // 2^7 J: sign bytes read as 2^-7 sgn
#pragma unroll
              for (int j = 0; j < NCH; ++j)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[q][j][v] = fmaf(wq, xv[u][j][v], acc[q][j][v]);
            }
        }
      }
      pk = pkn;
      jp = jpn;
    }

    // symplectic Euler: momentum with the old position, then position, then wall
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const int row = __ldg(a.grows + (size_t)grp * RW + q);
      if (row < 0) continue;
      const int ev = a.row_event ? __ldg(a.row_event + row) : 0;
      const float c0 = __ldg(a.c0_ev + ev);
      const float hi = __ldg(a.h + row);
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const size_t idx = (size_t)row * R + rep0 + 128 * j;
        const float4 xo = __ldg(reinterpret_cast<const float4*>(a.xin + idx));
        const float4 yo = *reinterpret_cast<const float4*>(a.y + idx);
        float xs[4] = {xo.x, xo.y, xo.z, xo.w}, ys[4] = {yo.x, yo.y, yo.z, yo.w};
        uint32_t sw = 0u;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          float x = xs[v], y = ys[v];
          float force = -pa * x + c0 * (acc[q][j][v] + hi);
          if (VARIANT == 0) force -= x * x * x;
          y = y + a.dt * force;
          x = x + a.dta0 * y;
          if (VARIANT != 0 && fabsf(x) > 1.f) {
            x = copysignf(1.f, x);
            y = 0.f;
          }
          xs[v] = x;
          ys[v] = y;
          if (use_sgn) sw |= sign_byte(x) << (8 * v);
        }
        if (use_sgn) *reinterpret_cast<uint32_t*>(a.sgn_out + idx) = sw;
        *reinterpret_cast<float4*>(a.xout + idx) = make_float4(xs[0], xs[1], xs[2], xs[3]);
        *reinterpret_cast<float4*>(a.y + idx) = make_float4(ys[0], ys[1], ys[2], ys[3]);
      }
    }
  }
}

template <int RW, int NCH, typename JT>
cudaError_t launch_t(int variant, const RwArgs& a, cudaStream_t s) {
  dim3 grid((a.ngroups + a.gpc - 1) / a.gpc, a.R / (128 * NCH));
  switch (variant) {
    case 0: k_step_rw<RW, NCH, 0, JT><<<grid, kRwBlock, 0, s>>>(a); break;
    case 1: k_step_rw<RW, NCH, 1, JT><<<grid, kRwBlock, 0, s>>>(a); break;
    default:
      if (a.sgn_in)
        k_step_rw<RW, NCH, 3, JT><<<grid, kRwBlock, 0, s>>>(a);
      else
        k_step_rw<RW, NCH, 2, JT><<<grid, kRwBlock, 0, s>>>(a);
      break;
  }
  return cudaGetLastError();
}

template <int RW, int NCH>
cudaError_t launch_j(int variant, int jbf16, const RwArgs& a, cudaStream_t s) {
  return jbf16 ? launch_t<RW, NCH, __nv_bfloat16>(variant, a, s)
               : launch_t<RW, NCH, float>(variant, a, s);
}

template <typename JT>
__global__ void k_fill_ejv(const JT* J, const int32_t* pos, int64_t count, JT* ejv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = pos[i];
    ejv[i] = p >= 0 ? J[p] : JT(0.f);
  }
}

}  // namespace

cudaError_t launch_step_rw(int variant, int jbf16, int rw, int nch, const RwArgs& a,
                           cudaStream_t s) {
  if (a.R % (128 * nch) != 0 || a.ngroups < 1 || a.gpc < 1) return cudaErrorInvalidValue;
  if (rw == 4) return nch == 2 ? launch_j<4, 2>(variant, jbf16, a, s) : launch_j<4, 1>(variant, jbf16, a, s);
  if (rw == 2) return nch == 2 ? launch_j<2, 2>(variant, jbf16, a, s) : launch_j<2, 1>(variant, jbf16, a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fill_ejv(const void* J, int jbf16, const int32_t* pos, int64_t count,
                            void* ejv, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((count + 255) / 256, 4096);
  if (jbf16)
    k_fill_ejv<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(J), pos,
                                                   count, static_cast<__nv_bfloat16*>(ejv));
  else
    k_fill_ejv<float><<<grid, 256, 0, s>>>(static_cast<const float*>(J), pos, count,
                                           static_cast<float*>(ejv));
  return cudaGetLastError();
}

SB_CHECK_READER(chk_read_rw)

}  // namespace sbd
