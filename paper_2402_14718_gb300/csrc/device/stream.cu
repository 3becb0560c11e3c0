// k_step_stream: one SB step (coupling product of Eq. 2 / 6 / 10, symplectic
// Euler update, inelastic wall) with the neighbour gather staged through
// shared memory by bulk asynchronous copies.
//
// Each CTA walks a contiguous chunk of rows, cut into blocks of kStreamBR rows.
// A block's neighbour columns form a sorted union list (padded to whole stages
// of kStreamSPS entries); every entry carries a mask of the block rows that
// use it. The producer warp copies, for every entry in use, the x row of that
// column (the W replicas of the current replica tile, 4W bytes) into one slot
// of a ring of `nst` stages, and the block's J values into one of two staging
// buffers; mbarriers with transaction counts signal arrival. Each consumer
// warp owns kStreamRW rows of the block and, entry by entry, multiplies the
// slot by the J value of each of its rows that uses the column. A column
// shared by several rows of the block is thus copied from L2 once, and read
// from shared memory once per warp instead of once per row.
//
// Accumulation order per (row, replica) is the row's CSR order (ascending
// column), one FMA per nonzero, as in k_step: both kernels give identical
// results.
//
// Every wait is bounded: after a.wait_ns (2 s by default; or once another
// warp has given up) a warp records a code in *err and returns; the producer
// first waits, again with a bound, for its copies still in flight. A test
// hook (a.skip_stage) makes CTA 0's producer leave one stage unissued -- no
// arrival and no copy, so nothing is in flight for it -- which runs the
// consumers' wait for that stage out.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "signs.cuh"

namespace sbd {
namespace {

constexpr unsigned long long kDrainNs = 200000000ull;   // 0.2 s
constexpr int kSmemBudgetCap = 232448;                  // 227 KB opt-in per block

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bytes (a multiple of 16) from global src (16-byte aligned) to shared dst
// (16-byte aligned); completion is counted on barrier bar
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The whole warp waits for the completion of phase parity `par` of `bar`.
// Returns false (the warp must leave) after limit_ns, or as soon as *err is set.
__device__ bool warp_wait(uint32_t bar, uint32_t par, int* err, int code,
                          unsigned long long limit_ns) {
  if (__all_sync(0xffffffffu, mbar_try(bar, par))) return true;
  const unsigned long long t0 = now_ns();
  for (uint32_t it = 1;; ++it) {
    if (__all_sync(0xffffffffu, mbar_try(bar, par))) return true;
    if ((it & 63) == 0) {
      int quit = 0;
      if ((threadIdx.x & 31) == 0) {
        if (*(volatile int*)err != 0) {
          quit = 1;
        } else if (now_ns() - t0 > limit_ns) {
          atomicCAS(err, 0, code);
          quit = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, quit, 0)) return false;
    }
  }
}

// Producer exit: wait (bounded, whatever *err says) until the copies of the
// last use of every ring stage and both J buffers have landed. A stage that
// was never issued (the test hook) is skipped: nothing of it is in flight.
__device__ void drain(uint32_t full0, int nst, int issued, int skipped,
                      unsigned long long limit_ns) {
  const unsigned long long lim = limit_ns < kDrainNs ? limit_ns : kDrainNs;
  const int first = issued > nst ? issued - nst : 0;
  for (int g = first; g < issued; ++g) {
    if (g == skipped) continue;
    const uint32_t bar = full0 + 8u * (uint32_t)(g % nst);
    const uint32_t par = (uint32_t)((g / nst) & 1);
    const unsigned long long t0 = now_ns();
    while (!__all_sync(0xffffffffu, mbar_try(bar, par))) {
      if (now_ns() - t0 > lim) break;
    }
  }
}

template <int PER>
struct Lane;
template <>
struct Lane<8> {  // replicas 4l..4l+3 and 128+4l..128+4l+3 of the tile
  static __device__ __forceinline__ void ld(const float* p, int l, float (&v)[8]) {
    const float4 a = *reinterpret_cast<const float4*>(p + 4 * l);
    const float4 b = *reinterpret_cast<const float4*>(p + 128 + 4 * l);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  static __device__ __forceinline__ void st(float* p, int l, const float (&v)[8]) {
    *reinterpret_cast<float4*>(p + 4 * l) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(p + 128 + 4 * l) = make_float4(v[4], v[5], v[6], v[7]);
  }
};
template <>
struct Lane<4> {  // replicas 4l..4l+3
  static __device__ __forceinline__ void ld(const float* p, int l, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p + 4 * l);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  static __device__ __forceinline__ void st(float* p, int l, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p + 4 * l) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Lane<2> {  // replicas 2l, 2l+1
  static __device__ __forceinline__ void ld(const float* p, int l, float (&v)[2]) {
    const float2 a = *reinterpret_cast<const float2*>(p + 2 * l);
    v[0] = a.x; v[1] = a.y;
  }
  static __device__ __forceinline__ void st(float* p, int l, const float (&v)[2]) {
    *reinterpret_cast<float2*>(p + 2 * l) = make_float2(v[0], v[1]);
  }
};

__device__ __forceinline__ float jget(const float* J, int i) { return J[i]; }
__device__ __forceinline__ float jget(const __nv_bfloat16* J, int i) {
  return __bfloat162float(J[i]);
}

template <int PER, int VARIANT, typename JT>
__global__ void __launch_bounds__(kStreamThreads, 1) k_step_stream(const StreamArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int W = 32 * PER;
  constexpr int SLOTB = W * 4;
  constexpr int SPS = kStreamSPS;
  constexpr int RW = kStreamRW;
  constexpr int PF = 8;                 // producer: stages of union entries loaded ahead
  constexpr int UB = PER == 8 ? 2 : 4;  // consumer: union entries read per batch
  constexpr size_t ESZ = sizeof(JT);
  const int nst = a.nst;
  unsigned char* ring = sm;
  unsigned char* jbuf = sm + (size_t)nst * SPS * SLOTB;
  uint32_t* meta = reinterpret_cast<uint32_t*>(jbuf + 2 * (size_t)a.jbuf_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(meta + (size_t)nst * SPS);
  const uint32_t full0 = saddr(bars);
  const uint32_t empty0 = full0 + 8u * (uint32_t)nst;
  const uint32_t jempty0 = empty0 + 8u * (uint32_t)nst;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; ++i) {
      mbar_init(full0 + 8u * i, 1);
      mbar_init(empty0 + 8u * i, kStreamWarps);
    }
    mbar_init(jempty0, kStreamWarps);
    mbar_init(jempty0 + 8u, kStreamWarps);
    mbar_fence_init();
  }
  __syncthreads();

  const int b0 = a.cta_blk0[blockIdx.x];
  const int nb = a.cta_blk0[blockIdx.x + 1] - b0;
  if (nb <= 0) return;
  const int4 first = a.blk[b0];
  const int E0 = first.y;
  const int s_tile = (a.blk[b0 + nb].y - E0) / SPS;  // ring stages per replica tile
  const int s_all = s_tile * a.tiles;

  if (warp == kStreamWarps) {
    // ------------------------------------------------------------ producer
    // queue of the union entries (one per lane) of stages g .. g + PF - 1
    int qc[PF];
    uint32_t qm[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      qc[j] = 0;
      qm[j] = 0u;
      if (j < s_all) {
        const int e = E0 + (j % s_tile) * SPS + lane;
        qc[j] = __ldg(a.ucol + e);
        qm[j] = __ldg(a.umask + e);
      }
    }
    int g = 0;  // stages issued
    bool ok = true;
    const int skip = blockIdx.x == 0 ? a.skip_stage : -1;
    int4 d0 = first, d1 = a.blk[b0 + 1];
    for (int t = 0; t < a.tiles && ok; ++t) {
      const float* xt = a.xin + (size_t)t * W;
      for (int bi = 0; bi < nb && ok; ++bi) {
        const int lb = t * nb + bi;
        const int jb = lb & 1;
        const int bn = bi + 1 < nb ? b0 + bi + 1 : b0;  // next block (next tile: first block)
        const int4 n0 = a.blk[bn], n1 = a.blk[bn + 1];
        if (lb >= 2 &&
            !warp_wait(jempty0 + 8u * jb, (uint32_t)(((lb >> 1) - 1) & 1), a.err, 1, a.wait_ns)) {
          ok = false;
          break;
        }
        const int nstg = (d1.y - d0.y) / SPS;
        for (int s = 0; s < nstg; ++s, ++g) {
          const int slot = g % nst;
          const int use = g / nst;
          if (use >= 1 &&
              !warp_wait(empty0 + 8u * slot, (uint32_t)((use - 1) & 1), a.err, 2, a.wait_ns)) {
            ok = false;
            break;
          }
          const int col = qc[0];
          const uint32_t m = qm[0];
#pragma unroll
          for (int j = 0; j < PF - 1; ++j) {
            qc[j] = qc[j + 1];
            qm[j] = qm[j + 1];
          }
          if (g + PF < s_all) {
            const int e = E0 + ((g + PF) % s_tile) * SPS + lane;
            qc[PF - 1] = __ldg(a.ucol + e);
            qm[PF - 1] = __ldg(a.umask + e);
          }
          if (g == skip) continue;  // test hook: this stage is never issued
          meta[slot * SPS + lane] = m;
          const unsigned cp = __ballot_sync(0xffffffffu, m != 0);
          const uint32_t jbytes = s == 0 ? (uint32_t)d0.w : 0u;
          const uint32_t bytes = (uint32_t)__popc(cp) * SLOTB + jbytes;
          __threadfence_block();
          __syncwarp();
          const uint32_t fb = full0 + 8u * slot;
          if (lane == 0) mbar_arrive_tx(fb, bytes);
          __syncwarp();
          if (m != 0)
            bulk_copy(saddr(ring + ((size_t)slot * SPS + lane) * SLOTB), xt + (size_t)col * a.R,
                      SLOTB, fb);
          if (lane == 0 && jbytes != 0)
            bulk_copy(saddr(jbuf + (size_t)jb * a.jbuf_bytes),
                      static_cast<const unsigned char*>(a.J) + (size_t)d0.z * ESZ, jbytes, fb);
        }
        d0 = n0;
        d1 = n1;
      }
    }
    drain(full0, nst, g, skip, a.wait_ns);
    return;
  }

  // -------------------------------------------------------------- consumers
  const int sh = warp * RW;
  const float pa = a.a0 - __ldg(a.sched + a.k);
  int4 d0 = first, d1 = a.blk[b0 + 1];
  int rj[RW];  // J offsets (inside the block's J span) of this warp's rows
#pragma unroll
  for (int q = 0; q < RW; ++q) {
    const int row = d0.x + sh + q;
    rj[q] = row < d1.x ? __ldg(a.rjo + row) : 0;
  }
  int g = 0;
  for (int t = 0; t < a.tiles; ++t) {
    for (int bi = 0; bi < nb; ++bi) {
      const int lb = t * nb + bi;
      const int jb = lb & 1;
      const int bn = bi + 1 < nb ? b0 + bi + 1 : b0;
      const int4 n0 = a.blk[bn], n1 = a.blk[bn + 1];
      const int r0 = d0.x, r1 = d1.x;
      // the next block's rows start where this block ends (or at the CTA's first row)
      const int nrow0 = bi + 1 < nb ? r1 : first.x;
      int rjn[RW];
#pragma unroll
      for (int q = 0; q < RW; ++q) {
        const int row = nrow0 + sh + q;
        rjn[q] = row < a.n ? __ldg(a.rjo + row) : 0;
      }
      const JT* jv = reinterpret_cast<const JT*>(jbuf + (size_t)jb * a.jbuf_bytes);
      int joff[RW];
      float xr[RW][PER], yr[RW][PER], acc[RW][PER], hq[RW];
      int evq[RW];
#pragma unroll
      for (int q = 0; q < RW; ++q) {
        const int row = r0 + sh + q;
        joff[q] = rj[q];
        hq[q] = 0.f;
        evq[q] = 0;
#pragma unroll
        for (int v = 0; v < PER; ++v) {
          acc[q][v] = 0.f;
          xr[q][v] = 0.f;
          yr[q][v] = 0.f;
        }
        if (row < r1) {
          const size_t idx = (size_t)row * a.R + (size_t)t * W;
          Lane<PER>::ld(a.xin + idx, lane, xr[q]);
          Lane<PER>::ld(a.y + idx, lane, yr[q]);
          hq[q] = __ldg(a.h + row);
          if (a.row_event) evq[q] = __ldg(a.row_event + row);
        }
      }
      for (int e = d0.y; e < d1.y; e += SPS, ++g) {
        const int slot = g % nst;
        const int use = g / nst;
        if (!warp_wait(full0 + 8u * slot, (uint32_t)(use & 1), a.err, 3, a.wait_ns)) return;
        const uint32_t mk = (meta[slot * SPS + lane] >> sh) & ((1u << RW) - 1u);
        unsigned act = __ballot_sync(0xffffffffu, mk != 0);
        const float* sb = reinterpret_cast<const float*>(ring + (size_t)slot * SPS * SLOTB);
        while (act) {
          int ks[UB];
          uint32_t ms[UB];
#pragma unroll
          for (int u = 0; u < UB; ++u) {
            ks[u] = 0;
            ms[u] = 0u;
            if (act) {
              ks[u] = __ffs(act) - 1;
              act &= act - 1;
              ms[u] = __shfl_sync(0xffffffffu, mk, ks[u]);
            }
          }
          float xs[UB][PER], wv[UB][RW];
#pragma unroll
          for (int u = 0; u < UB; ++u) Lane<PER>::ld(sb + ks[u] * W, lane, xs[u]);
#pragma unroll
          for (int u = 0; u < UB; ++u)
#pragma unroll
            for (int q = 0; q < RW; ++q) {
              wv[u][q] = 0.f;
              if (ms[u] & (1u << q)) wv[u][q] = jget(jv, joff[q]++);
            }
#pragma unroll
          for (int u = 0; u < UB; ++u) {
            if (VARIANT == 2) {
#pragma unroll
              for (int v = 0; v < PER; ++v) xs[u][v] = sgnf(xs[u][v]);
            }
#pragma unroll
            for (int q = 0; q < RW; ++q)
              if (ms[u] & (1u << q)) {
#pragma unroll
                for (int v = 0; v < PER; ++v) acc[q][v] = fmaf(wv[u][q], xs[u][v], acc[q][v]);
              }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8u * slot);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(jempty0 + 8u * jb);

      // symplectic Euler: momentum with the old position, then position, then wall
#pragma unroll
      for (int q = 0; q < RW; ++q) {
        const int row = r0 + sh + q;
        if (row >= r1) continue;
        const float c0 = __ldg(a.c0_ev + evq[q]);
#pragma unroll
        for (int v = 0; v < PER; ++v) {
          float x = xr[q][v], y = yr[q][v];
          float force = -pa * x + c0 * (acc[q][v] + hq[q]);
          if (VARIANT == 0) force -= x * x * x;
          y = y + a.dt * force;
          x = x + a.dta0 * y;
          if (VARIANT != 0 && fabsf(x) > 1.f) {
            x = copysignf(1.f, x);
            y = 0.f;
          }
          xr[q][v] = x;
          yr[q][v] = y;
        }
        const size_t idx = (size_t)row * a.R + (size_t)t * W;
        Lane<PER>::st(a.xout + idx, lane, xr[q]);
        Lane<PER>::st(a.y + idx, lane, yr[q]);
      }
      d0 = n0;
      d1 = n1;
#pragma unroll
      for (int q = 0; q < RW; ++q) rj[q] = rjn[q];
    }
  }
}

template <int PER, int VARIANT, typename JT>
cudaError_t launch_t(const StreamArgs& a, size_t smem, cudaStream_t s) {
  k_step_stream<PER, VARIANT, JT><<<a.grid, kStreamThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int PER, typename JT>
cudaError_t launch_v(int variant, const StreamArgs& a, size_t smem, cudaStream_t s) {
  switch (variant) {
    case 0: return launch_t<PER, 0, JT>(a, smem, s);
    case 1: return launch_t<PER, 1, JT>(a, smem, s);
    default: return launch_t<PER, 2, JT>(a, smem, s);
  }
}

template <int PER, int VARIANT, typename JT>
cudaError_t attr_t() {
  return cudaFuncSetAttribute(k_step_stream<PER, VARIANT, JT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudgetCap);
}

template <int PER, typename JT>
cudaError_t attr_v() {
  cudaError_t e = attr_t<PER, 0, JT>();
  if (e == cudaSuccess) e = attr_t<PER, 1, JT>();
  if (e == cudaSuccess) e = attr_t<PER, 2, JT>();
  return e;
}

}  // namespace

int stream_tile_width(int R) {
  if (R % 256 == 0) return 256;
  if (R % 128 == 0) return 128;
  if (R % 64 == 0) return 64;
  return 0;
}

size_t stream_smem(int W, int jbuf_bytes, int* nst_out) {
  const size_t per_stage = (size_t)kStreamSPS * W * 4 + (size_t)kStreamSPS * 4 + 16;
  const size_t fixed = 2 * (size_t)jbuf_bytes + 16;
  int nst = 0;
  if ((size_t)kSmemBudgetCap > fixed) nst = (int)(((size_t)kSmemBudgetCap - fixed) / per_stage);
  if (nst > 16) nst = 16;
  *nst_out = nst;
  if (nst < 2) return 0;
  return fixed + (size_t)nst * per_stage;
}

cudaError_t stream_prepare() {
  cudaError_t e = attr_v<8, float>();
  if (e == cudaSuccess) e = attr_v<8, __nv_bfloat16>();
  if (e == cudaSuccess) e = attr_v<4, float>();
  if (e == cudaSuccess) e = attr_v<4, __nv_bfloat16>();
  if (e == cudaSuccess) e = attr_v<2, float>();
  if (e == cudaSuccess) e = attr_v<2, __nv_bfloat16>();
  return e;
}

cudaError_t launch_step_stream(int variant, int jbf16, const StreamArgs& a, size_t smem,
                               cudaStream_t s) {
  switch (a.W) {
    case 256:
      return jbf16 ? launch_v<8, __nv_bfloat16>(variant, a, smem, s)
                   : launch_v<8, float>(variant, a, smem, s);
    case 128:
      return jbf16 ? launch_v<4, __nv_bfloat16>(variant, a, smem, s)
                   : launch_v<4, float>(variant, a, smem, s);
    case 64:
      return jbf16 ? launch_v<2, __nv_bfloat16>(variant, a, smem, s)
                   : launch_v<2, float>(variant, a, smem, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace sbd
