// Factored coupling product of the SB step (Eq. 2 / 6 / 10) for QUBOs whose
// couplings are mostly one weight shared by whole groups of rows.
//
// In the triplet QUBO of Eq. 13 every pair of triplets that share a hit and
// start on the same or adjacent layers is a conflict with the one weight w_c.
// Triplets holding hit h at position p form a group (h, p); triplets of groups
// (h, p) and (h, p') conflict exactly when |p - p'| <= 1. So the conflict part
// of J x is w (M^T W M) x with M the group incidence (three groups per
// triplet) and W the small position-coupling pattern, and the rest -- double
// counts of pairs sharing two hits, the consistent pairs (-1 instead of w_c)
// and the diagonal -- is an exact sparse residual formed on the host.
//
// One step is two launches:
//   k_fac_sum:  for each group block g (one hit), T_s = sum of x (or, for
//               dSB, of sgn x) over the block's members in slot s, then
//               U_s = sum_{s'} W[s][s'] T_{s'} for every slot whose U row a
//               factored row reads;
//   k_step_fac: for each row, f = jf * sum of its U rows + residual row . x,
//               then the fused symplectic-Euler update and wall.
// A row that the host found cheaper in its plain CSR form has no U rows and
// its whole CSR row as residual, so one kernel serves both kinds of rows.
//
// Layout: lane l of a G-lane row group covers, for FP32 state, the replicas
// tile0 + 4 l + 4 G j + v (j < NCH, v < 4), i.e. 16-byte chunks strided by the
// group; for dSB sign bytes the 8 replicas tile0 + 8 l + v (one 8-byte load
// per neighbour). U rows use the same replica layout: FP32 for aSB / bSB; for
// dSB BF16 sums of 2^-7 sgn (exact while no U element sums more than 256
// members), else FP32 sums (the dSB kernels' NCH = 2 instances; NCH has no
// other meaning there).
//
// Every sum is formed in a fixed order (members by slot and row, residual in
// column order), so results are reproducible. For dSB with weights that are
// multiples of 1/4 every partial sum is exact and the step equals the
// CSR-order kernels bit for bit; for aSB / bSB the rounding order differs from
// the CSR order (per-step agreement to ~1e-6 relative).
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "signs.cuh"

namespace sbd {
namespace {

constexpr int kFacBlock = 128;
// dSB: replicas per lane (measured on the 512-event batch against 16 per lane,
// and against requesting the U rows and own x, y before the residual walk:
// both cost occupancy and were slower)
constexpr int kSgnPer = 8;

// N 32-bit words loaded or stored as one vector (N = 2 or 4)
template <int N>
struct Words;
template <>
struct Words<2> {
  uint32_t w[2];
  __device__ __forceinline__ void ldg(const void* p) {
    const uint2 t = __ldg(static_cast<const uint2*>(p));
    w[0] = t.x;
    w[1] = t.y;
  }
  __device__ __forceinline__ void st(void* p) const {
    *static_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  }
};
template <>
struct Words<4> {
  uint32_t w[4];
  __device__ __forceinline__ void ldg(const void* p) {
    const uint4 t = __ldg(static_cast<const uint4*>(p));
    w[0] = t.x;
    w[1] = t.y;
    w[2] = t.z;
    w[3] = t.w;
  }
  __device__ __forceinline__ void st(void* p) const {
    *static_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  }
};

__device__ __forceinline__ unsigned lane_group_mask(int G) {
  const int lane = threadIdx.x & 31;
  return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// One member's values at this lane's replicas, as loaded: FP32 chunks
// (MODE 0) or 16 sign bytes (MODE 1, unpacked to 2^-7 sgn only when added).
template <int MODE, int NCH>
struct Chunk;
template <int NCH>
struct Chunk<0, NCH> {
  static constexpr int P = 4 * NCH;
  float4 t[NCH];
  __device__ __forceinline__ void load(const FacSumArgs& a, size_t off, int G, int row) {
#pragma unroll
    for (int j = 0; j < NCH; ++j)
      t[j] = __ldg(reinterpret_cast<const float4*>(a.xin + (size_t)row * a.R + off) + G * j);
  }
  __device__ __forceinline__ void add_to(float (&u)[P]) const {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      u[4 * j] += t[j].x;
      u[4 * j + 1] += t[j].y;
      u[4 * j + 2] += t[j].z;
      u[4 * j + 3] += t[j].w;
    }
  }
};
template <int NCH>
struct Chunk<1, NCH> {
  static constexpr int P = kSgnPer;
  Words<P / 4> t;
  __device__ __forceinline__ void load(const FacSumArgs& a, size_t off, int, int row) {
    t.ldg(a.sgn_in + (size_t)row * a.R + off);
  }
  __device__ __forceinline__ void add_to(float (&u)[P]) const {
#pragma unroll
    for (int k = 0; k < P; ++k) u[k] += scaled_sign_of_byte(t.w[k >> 2], k & 3);
  }
};

// Adds a member in slot s2 to every U_s it couples to (s2 is the same for the
// whole lane group, so the branches do not diverge inside it).
template <int K, typename CH>
__device__ __forceinline__ void add_member(float (&U)[K][CH::P], const CH& v, int s2,
                                           uint32_t couple) {
#pragma unroll
  for (int s = 0; s < K; ++s)
    if ((couple >> (4 * s + s2)) & 1u) v.add_to(U[s]);
}

// Write the K U rows of block g from the sums U (for every slot in use).
template <int MODE, int NCH, int K, int P>
__device__ __forceinline__ void store_u(const FacSumArgs& a, int g, size_t off, int G,
                                        const float (&U)[K][P]) {
#pragma unroll
  for (int s = 0; s < K; ++s) {
    int u = __ldg(a.gout + (size_t)g * K + s);
    if (u < 0) continue;
    u = chk_idx(u, a.urows, kChkURow);
    if (MODE == 0) {
      float4* p = reinterpret_cast<float4*>(static_cast<float*>(a.U) + (size_t)u * a.R + off);
#pragma unroll
      for (int j = 0; j < NCH; ++j)
        p[G * j] = make_float4(U[s][4 * j], U[s][4 * j + 1], U[s][4 * j + 2], U[s][4 * j + 3]);
    } else if (NCH == 2) {
      // dSB, blocks of more than 256 members: FP32 sums of 2^-7 sgn (exact)
      float4* p = reinterpret_cast<float4*>(static_cast<float*>(a.U) + (size_t)u * a.R + off);
#pragma unroll
      for (int h = 0; h < P / 4; ++h)
        p[h] = make_float4(U[s][4 * h], U[s][4 * h + 1], U[s][4 * h + 2], U[s][4 * h + 3]);
    } else {
      // sums of 2^-7 sgn of at most 256 members: exact in BF16 (the top half of the FP32 word)
      uint16_t* p = static_cast<uint16_t*>(a.U) + (size_t)u * a.R + off;
#pragma unroll
      for (int h = 0; h < P / 8; ++h) {
        Words<4> w;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          w.w[k] = (__float_as_uint(U[s][8 * h + 2 * k]) >> 16) |
                   (__float_as_uint(U[s][8 * h + 2 * k + 1]) & 0xffff0000u);
        w.st(p + 8 * h);
      }
    }
  }
}

// Lane l's P values of slot s of scratch slot c (the lane's own replicas).
template <int MODE, int NCH, int P>
__device__ __forceinline__ size_t scr_index(const FacSumArgs& a, int c, int s, size_t off, int G,
                                            int v) {
  const size_t base = ((size_t)c * a.K + s) * a.R + off;
  return MODE == 0 ? base + 4 * G * (v >> 2) + (v & 3) : base + v;
}

// residency bounds (CTAs of 128 threads per SM). dSB, measured on the
// 512-event batch: 12 for the row step (40 registers) and 10 for the group
// sums (48) beat the compiler's unbounded 48 / 64 registers (1.92 against
// 2.03 ms per step). The FP32 forms: the bounds that give the compiler's own
// unbounded register counts (about 48 / 56 registers with one 16-byte chunk per
// lane, 64 / 72 with two).
template <int MODE, int NCH>
struct FacMinBlocks {
  static constexpr int sum = NCH == 2 ? 7 : 9, step = NCH == 2 ? 8 : 9;
};
#ifndef SB_FAC_DSB_STEP_MINB
#define SB_FAC_DSB_STEP_MINB 12
#endif
template <int NCH>
struct FacMinBlocks<1, NCH> {
  static constexpr int sum = 10, step = SB_FAC_DSB_STEP_MINB;
};

template <int MODE, int NCH, int K>
__global__ void __launch_bounds__(kFacBlock, (FacMinBlocks<MODE, NCH>::sum)) k_fac_sum(const FacSumArgs a) {
  using C = Chunk<MODE, NCH>;
  constexpr int P = C::P;
  const int G = a.G;
  const int gq = threadIdx.x / G;
  const int l = threadIdx.x - gq * G;
  const int it = blockIdx.x * (kFacBlock / G) + gq;
  if (it >= a.nitems) return;  // the whole lane group leaves together
  const unsigned mask = lane_group_mask(G);
  const size_t off = MODE == 0 ? (size_t)blockIdx.y * (4 * G * NCH) + 4 * l
                               : (size_t)blockIdx.y * (kSgnPer * G) + kSgnPer * l;
  const int4 item = __ldg(a.item + it);
  const int g = item.x;
  // slot boundaries of the block's members (members grouped by slot)
  int bnd[K + 1];
#pragma unroll
  for (int s = 0; s <= K; ++s) bnd[s] = __ldg(a.gseg + (size_t)g * K + s);
  float U[K][P];
#pragma unroll
  for (int s = 0; s < K; ++s)
#pragma unroll
    for (int v = 0; v < P; ++v) U[s][v] = 0.f;
  // this item's members in one pass, G entries per load, four rows in flight;
  // each lane's entry carries its row and slot, broadcast by shuffles
  for (int mb = item.y; mb < item.z; mb += G) {
    const int cnt = min(G, item.z - mb);
    int mr = 0, ms = 0;
    if (l < cnt) {
      const int t = mb + l;
      mr = chk_idx(__ldg(a.gmem + t), a.n, kChkMember);
#pragma unroll
      for (int s = 1; s < K; ++s) ms += t >= bnd[s] ? 1 : 0;
    }
    int q = 0;
    for (; q + 4 <= cnt; q += 4) {
      int r[4], sl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        r[u] = __shfl_sync(mask, mr, q + u, G);
        sl[u] = __shfl_sync(mask, ms, q + u, G);
      }
      C v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u].load(a, off, G, r[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) add_member<K, C>(U, v[u], sl[u], a.couple);
    }
    for (; q < cnt; ++q) {
      const int r0 = __shfl_sync(mask, mr, q, G), s0 = __shfl_sync(mask, ms, q, G);
      C v0;
      v0.load(a, off, G, r0);
      add_member<K, C>(U, v0, s0, a.couple);
    }
  }
  if (item.w < 0) {  // the whole block in one item
    store_u<MODE, NCH, K, P>(a, g, off, G, U);
    return;
  }
  // one chunk of a split block: its sums to the scratch slot; the chunk that
  // finishes last adds every chunk's slot in chunk order (a fixed order, so
  // the result does not depend on which chunk finishes last)
#pragma unroll
  for (int s = 0; s < K; ++s)
#pragma unroll
    for (int v = 0; v < P; ++v) a.scratch[scr_index<MODE, NCH, P>(a, item.w, s, off, G, v)] = U[s][v];
  __threadfence();
  __syncwarp(mask);
  int last = 0;
  const int nc = __ldg(a.gnc + g);
  int* const cnt = a.cnt + (size_t)g * a.tiles + blockIdx.y;  // one counter per replica tile
  if (l == 0) last = atomicAdd(cnt, 1) == nc - 1;
  last = __shfl_sync(mask, last, 0, G);
  if (!last) return;
  __threadfence();
  const int c0 = __ldg(a.gscr0 + g);
#pragma unroll
  for (int s = 0; s < K; ++s)
#pragma unroll
    for (int v = 0; v < P; ++v) U[s][v] = 0.f;
  for (int c = 0; c < nc; ++c)
#pragma unroll
    for (int s = 0; s < K; ++s)
#pragma unroll
      for (int v = 0; v < P; ++v) U[s][v] += __ldcg(a.scratch + scr_index<MODE, NCH, P>(a, c0 + c, s, off, G, v));
  store_u<MODE, NCH, K, P>(a, g, off, G, U);
  if (l == 0) *cnt = 0;  // ready for the next launch
}

__device__ __forceinline__ float jv(const float* J, int p) { return __ldg(J + p); }
__device__ __forceinline__ float jv(const __nv_bfloat16* J, int p) {
  return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(J) + p) << 16);
}
// value t of a row head's J part (words from kFacHead + kFacHeadU on)
template <typename JT>
__device__ __forceinline__ float head_j(const uint32_t* hd, int t) {
  const uint32_t* p = hd + kFacHead + kFacHeadU;
  if (sizeof(JT) == 4) return __uint_as_float(__ldg(p + t));
  return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p) + t) << 16);
}

__global__ void k_fac_head(const FacHeadArgs a) {
  const int HW = fac_head_words(a.jbytes);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)a.n * HW) return;
  const int64_t row = t / HW;
  const int w = (int)(t - row * HW);
  const int p0 = a.rrowptr[row], L = a.rrowptr[row + 1] - p0;
  uint32_t v = 0;
  if (w < kFacHead) {
    v = w < L ? (uint32_t)a.rcol[p0 + w] : 0u;
  } else if (w < kFacHead + kFacHeadU) {
    const int s = w - kFacHead;
    v = s < a.K ? (uint32_t)a.uidx[row * a.K + s] : 0xffffffffu;
  } else if (a.jbytes == 4) {
    const int e = w - kFacHead - kFacHeadU;
    v = e < L ? static_cast<const uint32_t*>(a.rJ)[p0 + e] : 0u;
  } else {
    const int e = 2 * (w - kFacHead - kFacHeadU);
    const uint16_t* J = static_cast<const uint16_t*>(a.rJ);
    v = (e < L ? J[p0 + e] : 0u) | (e + 1 < L ? (uint32_t)J[p0 + e + 1] << 16 : 0u);
  }
  a.head[t] = v;
}

// Adds cnt residual entries (lane q of the lane group holds column mc and
// weight mw of entry q) to this lane's replicas, four neighbour rows in flight.
template <int MODE, int NCH, int P>
__device__ __forceinline__ void walk_entries(float (&acc)[P], int cnt, int mc, float mw,
                                             unsigned mask, int G, const float* xin,
                                             const uint8_t* sgn_in, size_t off, int R) {
  int q = 0;
  for (; q + 4 <= cnt; q += 4) {
    int c[4];
    float w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c[u] = __shfl_sync(mask, mc, q + u, G);
      w[u] = __shfl_sync(mask, mw, q + u, G);
    }
    if (MODE == 0) {
      float4 t[4][NCH];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < NCH; ++j)
          t[u][j] = __ldg(reinterpret_cast<const float4*>(xin + (size_t)c[u] * R + off) + G * j);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
          acc[4 * j] = fmaf(w[u], t[u][j].x, acc[4 * j]);
          acc[4 * j + 1] = fmaf(w[u], t[u][j].y, acc[4 * j + 1]);
          acc[4 * j + 2] = fmaf(w[u], t[u][j].z, acc[4 * j + 2]);
          acc[4 * j + 3] = fmaf(w[u], t[u][j].w, acc[4 * j + 3]);
        }
    } else {
      Words<kSgnPer / 4> t[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) t[u].ldg(sgn_in + (size_t)c[u] * R + off);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < kSgnPer && v < P; ++v)
          acc[v] = fmaf(w[u], scaled_sign_of_byte(t[u].w[v >> 2], v & 3), acc[v]);
    }
  }
  for (; q < cnt; ++q) {
    const int c = __shfl_sync(mask, mc, q, G);
    const float w = __shfl_sync(mask, mw, q, G);
    if (MODE == 0) {
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(xin + (size_t)c * R + off) + G * j);
        acc[4 * j] = fmaf(w, t.x, acc[4 * j]);
        acc[4 * j + 1] = fmaf(w, t.y, acc[4 * j + 1]);
        acc[4 * j + 2] = fmaf(w, t.z, acc[4 * j + 2]);
        acc[4 * j + 3] = fmaf(w, t.w, acc[4 * j + 3]);
      }
    } else {
      Words<kSgnPer / 4> t;
      t.ldg(sgn_in + (size_t)c * R + off);
#pragma unroll
      for (int v = 0; v < kSgnPer && v < P; ++v)
        acc[v] = fmaf(w, scaled_sign_of_byte(t.w[v >> 2], v & 3), acc[v]);
    }
  }
}

// One U row of this lane: FP32 (NCH float4) or BF16 sums of 2^-7 sgn (two uint4)
template <int MODE, int NCH>
struct URow;
template <int NCH>
struct URow<0, NCH> {
  float4 t[NCH];
  __device__ __forceinline__ void load(const void* U, size_t base, int G) {
#pragma unroll
    for (int j = 0; j < NCH; ++j)
      t[j] = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(U) + base) + G * j);
  }
  __device__ __forceinline__ void add_to(float (&fu)[4 * NCH]) const {
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      fu[4 * j] += t[j].x;
      fu[4 * j + 1] += t[j].y;
      fu[4 * j + 2] += t[j].z;
      fu[4 * j + 3] += t[j].w;
    }
  }
};
template <>
struct URow<1, 2> {  // dSB with FP32 U rows
  float4 t[kSgnPer / 4];
  __device__ __forceinline__ void load(const void* U, size_t base, int) {
#pragma unroll
    for (int h = 0; h < kSgnPer / 4; ++h)
      t[h] = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(U) + base) + h);
  }
  __device__ __forceinline__ void add_to(float (&fu)[kSgnPer]) const {
#pragma unroll
    for (int h = 0; h < kSgnPer / 4; ++h) {
      fu[4 * h] += t[h].x;
      fu[4 * h + 1] += t[h].y;
      fu[4 * h + 2] += t[h].z;
      fu[4 * h + 3] += t[h].w;
    }
  }
};
template <int NCH>
struct URow<1, NCH> {
  Words<4> t[kSgnPer / 8];  // kSgnPer BF16 sums
  __device__ __forceinline__ void load(const void* U, size_t base, int) {
    const uint16_t* p = static_cast<const uint16_t*>(U) + base;
#pragma unroll
    for (int h = 0; h < kSgnPer / 8; ++h) t[h].ldg(p + 8 * h);
  }
  __device__ __forceinline__ void add_to(float (&fu)[kSgnPer]) const {
#pragma unroll
    for (int h = 0; h < kSgnPer / 8; ++h)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        fu[8 * h + 2 * k] += __uint_as_float(t[h].w[k] << 16);
        fu[8 * h + 2 * k + 1] += __uint_as_float(t[h].w[k] & 0xffff0000u);
      }
  }
};

// VARIANT 0 aSB, 1 bSB (MODE 0: FP32 x), 2 dSB (MODE 1: sign bytes)
template <int VARIANT, int MODE, int NCH, int K, typename JT>
__global__ void __launch_bounds__(kFacBlock, (FacMinBlocks<MODE, NCH>::step)) k_step_fac(const FacStepArgs a) {
  constexpr int P = MODE == 0 ? 4 * NCH : kSgnPer;
  constexpr int NV = P / 4;  // float4 of own x (and y) per lane
  const int G = a.G;
  const int gq = threadIdx.x / G;
  const int l = threadIdx.x - gq * G;
  const int row = blockIdx.x * (kFacBlock / G) + gq;
  if (row >= a.n) return;
  const unsigned mask = lane_group_mask(G);
  const int R = a.R;
  const size_t off = MODE == 0 ? (size_t)blockIdx.y * (4 * G * NCH) + 4 * l
                               : (size_t)blockIdx.y * (kSgnPer * G) + kSgnPer * l;
  const size_t idx = (size_t)row * R + off;
  const JT* J = static_cast<const JT*>(a.rJ);
  // the row's own x and y and its U rows are read after the residual walk:
  // ask for them in L2 now, so that those loads do not wait on HBM
#pragma unroll
  for (int j = 0; j < P / 4; ++j) {
    const size_t o = MODE == 0 ? idx + 4 * G * j : idx + 4 * j;
    prefetch_l2(a.xin + o);
    prefetch_l2(a.y + o);
  }
  constexpr int HW = fac_head_words(sizeof(JT));
  const uint32_t* hd = a.head + (size_t)row * HW;
  int us[K];
#pragma unroll
  for (int s = 0; s < K; ++s) {
    us[s] = (int)__ldg(hd + kFacHead + s);
    if (us[s] >= 0) us[s] = chk_idx(us[s], a.urows, kChkURow);
    if (us[s] >= 0)
      prefetch_l2(static_cast<const char*>(a.U) + ((size_t)us[s] * R + off) * (MODE == 0 || NCH == 2 ? 4 : 2));
  }
  int p0 = __ldg(a.rrowptr + row), p1 = __ldg(a.rrowptr + row + 1);
  chk_rows(p0, p1, a.rnnz);

  // residual row, in column order: its first kFacHead entries from the head,
  // the rest from the residual CSR
  float acc[P];
#pragma unroll
  for (int v = 0; v < P; ++v) acc[v] = 0.f;
  const int nh = min(p1 - p0, kFacHead);
  for (int hb = 0; hb < nh; hb += G) {
    const int cnt = min(G, nh - hb);
    int mc = 0;
    float mw = 0.f;
    if (l < cnt) {
      mc = chk_idx((int)__ldg(hd + hb + l), a.n, kChkCol);
      mw = head_j<JT>(hd, hb + l);
      if (MODE == 1) mw *= kSignScale;  // 2^7 J: sign bytes read as 2^-7 sgn
    }
    walk_entries<MODE, NCH, P>(acc, cnt, mc, mw, mask, G, a.xin, a.sgn_in, off, R);
  }
  for (int pb = p0 + kFacHead; pb < p1; pb += G) {
    const int cnt = min(G, p1 - pb);
    int mc = 0;
    float mw = 0.f;
    if (l < cnt) {
      mc = chk_idx(__ldg(a.rcol + pb + l), a.n, kChkCol);
      mw = jv(J, pb + l);
      if (MODE == 1) mw *= kSignScale;
    }
    walk_entries<MODE, NCH, P>(acc, cnt, mc, mw, mask, G, a.xin, a.sgn_in, off, R);
  }
  // the factored part: sum of this row's U rows (none for a plain row)
  bool any = false;
  float fu[P];
#pragma unroll
  for (int v = 0; v < P; ++v) fu[v] = 0.f;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    if (us[s] < 0) continue;
    any = true;
    URow<MODE, NCH> ur;
    ur.load(a.U, (size_t)us[s] * R + off, G);
    ur.add_to(fu);
  }
  // dSB: U holds sums of 2^-7 sgn, so the scale is 2^7 jf (exact)
  const float jf = MODE == 1 ? a.jf * kSignScale : a.jf;
  if (any) {
#pragma unroll
    for (int v = 0; v < P; ++v) acc[v] = fmaf(jf, fu[v], acc[v]);
  }

  // symplectic Euler: momentum with the old position, then position, then wall
  const float pa = a.a0 - __ldg(a.sched + a.k);
  const int ev = a.row_event ? __ldg(a.row_event + row) : 0;
  const float c0 = __ldg(a.c0_ev + ev);
  const float hi = __ldg(a.h + row);
  Words<kSgnPer / 4> sw;  // dSB: the new sign bytes
#pragma unroll
  for (int k = 0; k < kSgnPer / 4; ++k) sw.w[k] = 0u;
  const bool inplace = a.xout == a.xin;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const size_t o = MODE == 0 ? idx + 4 * G * j : idx + 4 * j;
    const float4 xo = __ldg(reinterpret_cast<const float4*>(a.xin + o));
    const float4 yo = *reinterpret_cast<const float4*>(a.y + o);
    float xs[4] = {xo.x, xo.y, xo.z, xo.w}, ys[4] = {yo.x, yo.y, yo.z, yo.w};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float x = xs[v], y = ys[v];
      float force = -pa * x + c0 * (acc[4 * j + v] + hi);
      if (VARIANT == 0) force -= x * x * x;
      y = y + a.dt * force;
      x = x + a.dta0 * y;
      if (VARIANT != 0 && fabsf(x) > 1.f) {
        x = copysignf(1.f, x);
        y = 0.f;
      }
      xs[v] = x;
      ys[v] = y;
      if (MODE == 1 && j < kSgnPer / 4) sw.w[j] |= sign_byte(x) << (8 * v);
    }
    // a spin that stays on the wall keeps x = +-1, y = 0: nothing to write back
    // where the value is updated in place (y always; x on the dSB path)
    const float4 xn = make_float4(xs[0], xs[1], xs[2], xs[3]);
    const float4 yn = make_float4(ys[0], ys[1], ys[2], ys[3]);
    if (!inplace || bits_differ(xo, xn)) *reinterpret_cast<float4*>(a.xout + o) = xn;
    if (bits_differ(yo, yn)) *reinterpret_cast<float4*>(a.y + o) = yn;
  }
  if (MODE == 1) sw.st(a.sgn_out + idx);
}

template <int MODE, int NCH, int K>
cudaError_t launch_sum_k(const FacSumArgs& a, cudaStream_t s) {
  if (a.nitems <= 0) return cudaSuccess;
  const int per = kFacBlock / a.G;
  dim3 grid((a.nitems + per - 1) / per, a.tiles);
  k_fac_sum<MODE, NCH, K><<<grid, kFacBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <int MODE, int NCH>
cudaError_t launch_sum_n(const FacSumArgs& a, cudaStream_t s) {
  switch (a.K) {
    case 1: return launch_sum_k<MODE, NCH, 1>(a, s);
    case 2: return launch_sum_k<MODE, NCH, 2>(a, s);
    case 3: return launch_sum_k<MODE, NCH, 3>(a, s);
    case 4: return launch_sum_k<MODE, NCH, 4>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int VARIANT, int MODE, int NCH, int K, typename JT>
cudaError_t launch_step_k(const FacStepArgs& a, cudaStream_t s) {
  const int per = kFacBlock / a.G;
  dim3 grid((a.n + per - 1) / per, a.tiles);
  k_step_fac<VARIANT, MODE, NCH, K, JT><<<grid, kFacBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <int VARIANT, int MODE, int NCH, typename JT>
cudaError_t launch_step_n(const FacStepArgs& a, cudaStream_t s) {
  switch (a.K) {
    case 1: return launch_step_k<VARIANT, MODE, NCH, 1, JT>(a, s);
    case 2: return launch_step_k<VARIANT, MODE, NCH, 2, JT>(a, s);
    case 3: return launch_step_k<VARIANT, MODE, NCH, 3, JT>(a, s);
    case 4: return launch_step_k<VARIANT, MODE, NCH, 4, JT>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename JT>
cudaError_t launch_step_j(int variant, const FacStepArgs& a, cudaStream_t s) {
  if (variant == 2) return a.NCH == 2 ? launch_step_n<2, 1, 2, JT>(a, s) : launch_step_n<2, 1, 1, JT>(a, s);
  if (a.NCH == 2)
    return variant == 0 ? launch_step_n<0, 0, 2, JT>(a, s) : launch_step_n<1, 0, 2, JT>(a, s);
  return variant == 0 ? launch_step_n<0, 0, 1, JT>(a, s) : launch_step_n<1, 0, 1, JT>(a, s);
}

}  // namespace

bool fac_tiling(int variant, int R, int* G, int* NCH, int* tiles) {
  if (R < 1) return false;
  if (variant == 2) {
    if (R % kSgnPer) return false;
    const int C = R / kSgnPer;
    if (C <= 32 && (C & (C - 1)) == 0) {
      *G = C;
      *NCH = 1;
      *tiles = 1;
      return true;
    }
    if (C % 32 == 0) {
      *G = 32;
      *NCH = 1;
      *tiles = C / 32;
      return true;
    }
    return false;
  }
  if (R % 4) return false;
  const int C = R / 4;
  if (C <= 32 && (C & (C - 1)) == 0) {
    *G = C;
    *NCH = 1;
    *tiles = 1;
    return true;
  }
  if (C % 64 == 0) {
    *G = 32;
    *NCH = 2;
    *tiles = C / 64;
    return true;
  }
  if (C % 32 == 0) {
    *G = 32;
    *NCH = 1;
    *tiles = C / 32;
    return true;
  }
  return false;
}

cudaError_t launch_fac_head(const FacHeadArgs& a, cudaStream_t s) {
  const int64_t total = (int64_t)a.n * fac_head_words(a.jbytes);
  if (total <= 0) return cudaSuccess;
  k_fac_head<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fac_sum(int variant, const FacSumArgs& a, cudaStream_t s) {
  if (variant == 2) return a.NCH == 2 ? launch_sum_n<1, 2>(a, s) : launch_sum_n<1, 1>(a, s);
  return a.NCH == 2 ? launch_sum_n<0, 2>(a, s) : launch_sum_n<0, 1>(a, s);
}

cudaError_t launch_step_fac(int variant, int jbf16, const FacStepArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  return jbf16 ? launch_step_j<__nv_bfloat16>(variant, a, s) : launch_step_j<float>(variant, a, s);
}

SB_CHECK_READER(chk_read_factor)

}  // namespace sbd
