// Internal interface between the C ABI (api.cu) and the device kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "checks.cuh"

namespace sbd {

// Replica tiling of the N x R state: each row is handled by a group of G
// threads (G a power of two <= 32); a thread covers NCH chunks of V
// consecutive replicas, chunks strided by G so a group reads contiguous bytes.
struct Tiling {
  int V;      // replicas per chunk: 4 (float4) or 1
  int G;      // threads per row
  int NCH;    // chunks per thread per replica tile: 1, 2 or 4
  int tiles;  // replica tiles (grid.y)
  int C;      // chunks per row = R / V
};
Tiling make_tiling(int R);
// Tiling with a fixed replica-tile width RT (a multiple of 4 dividing R, RT <= 128):
// V = 4, G = RT / 4 threads per row, one chunk per thread, R / RT tiles.
Tiling make_tiling_rt(int R, int RT);
// dSB with int8 signs, 16 replicas per lane: valid when R / 16 is a power of two <= 32.
bool dsb16_ok(int R);
// rows per CTA of k_step_dsb16 for a step's rows-per-CTA setting rpc
int dsb16_rows_per_cta(int rpc);
Tiling make_tiling_dsb16(int R);

struct StepArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const void* J;          // float or __nv_bfloat16, -b/4
  const float* h;         // FP32 field
  const int32_t* row_event;  // event of each row (NULL: single event)
  const float* c0_ev;     // per-event c0
  const float* sched;     // a_k, device
  int32_t k;              // step index into sched
  float a0, dt, dta0;     // dta0 = fp32(dt * a0)
  const float* xin;
  float* xout;
  float* y;
  int32_t n, R;
  int32_t G;
  int32_t rpc;            // rows per CTA: a CTA walks rows [b * rpc, (b + 1) * rpc)
  float* ytil;            // optional: momentum after the update, before the wall [n x R]
  uint8_t* mask;          // optional: 1 where the wall fired [n x R]
  float* frec;            // optional (with ytil): the coupling sum J g(x) [n x R]
  int32_t r1_lanes = 0;   // R = 1: lanes per row (8, 16, 32: k_step_r1g; else one thread per row)
  const uint8_t* sgn_in;  // dSB: sign bytes of x_k [n x R] gathered instead of x (NULL: use x)
  uint8_t* sgn_out;       // dSB: sign bytes of x_{k+1}, written with x_{k+1} (may be NULL)
  // k_step_dsb16: CTA b takes row chunk cta_order[b] (chunks of
  // dsb16_rows_per_cta(rpc) rows, heaviest first); NULL: chunk b
  const int32_t* cta_order = nullptr;
  int32_t unroll;         // neighbours in flight per thread (4)
  int32_t tile0;          // first replica tile of this launch (sequential replica groups)
  int64_t nnz = INT64_MAX;  // CSR entries (the bounds-checked build tests rowptr against it)
};

cudaError_t launch_step(int variant, int jbf16, const Tiling& t, const StepArgs& a,
                        cudaStream_t s);

// Row-block tiling of the coupling product: rows are cut into blocks whose
// union of neighbour rows ("ucol") fits kTileUCap; each CTA stages that union
// for one 32-replica tile in shared memory and computes its block from there.
constexpr int kTileRT = 32;        // replicas per tile
constexpr int kTileUCap = 512;     // union rows per block (64 KB of FP32 x)
constexpr int kTileNzCap = 4096;   // nonzeros per block
constexpr int kTileRowCap = 256;   // rows per block

struct TiledArgs {
  const int32_t* blk_row0;   // [nb + 1] first row of each block
  const int32_t* blk_u0;     // [nb + 1] offset of each block's union in ucol
  const int32_t* ucol;       // union rows (global row ids), ascending within a block
  const uint16_t* own;       // [n] local index of row i inside its block's union
  const int32_t* rowptr;     // CSR row pointers (global)
  const void* tz;            // per nonzero: packed (local index, J): u32 for BF16, u64 for FP32
  const float* h;
  const int32_t* row_event;
  const float* c0_ev;
  const float* sched;
  int32_t k;
  float a0, dt, dta0;
  const float* xin;
  float* xout;
  float* y;
  int32_t n, R, nb;
};

cudaError_t launch_step_tiled(int variant, int jbf16, const TiledArgs& a, cudaStream_t s);
// tz[p] = packed (lidx[p], J[p]) (u32 for BF16 J, u64 for FP32 J)
cudaError_t launch_pack_tz(const void* J, int jbf16, const uint16_t* lidx, int64_t nnz, void* tz,
                           cudaStream_t s);

cudaError_t launch_init(float* x, float* y, const int32_t* row_event, const int32_t* ev_row0,
                        int32_t n, int32_t R, uint64_t seed, cudaStream_t s);
// s[i] = sign byte of x[i]: 0x3C, 0xBC, 0x00 for x > 0, x < 0, x = 0 (signs.cuh)
cudaError_t launch_signs(const float* x, uint8_t* s, size_t count, cudaStream_t st);
// blocks of the untiled step kernel resident per SM for this tiling and unroll
int step_blocks_per_sm(int variant, int jbf16, const Tiling& t, int unroll);

cudaError_t launch_linear_schedule(float* sched, int32_t steps, double a0, cudaStream_t s);

cudaError_t launch_set_c0(float* c0_ev, const double* c0_auto, double c0, int32_t E,
                          cudaStream_t s);

// QUBO -> Ising in FP64 (per row), then per-event reductions.
cudaError_t launch_convert(const int32_t* rowptr, const int32_t* col, const double* qval,
                           const double* qlin, int32_t n, void* J, int jbf16, double* h64,
                           float* h32, double* row_off, double* row_sq, cudaStream_t s);
cudaError_t launch_event_stats(const double* row_off, const double* row_sq,
                               const int32_t* ev_row0, int32_t E, double* offset,
                               double* sigma, double* c0_auto, cudaStream_t s);

struct EnergyArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const double* qval;
  const double* qlin;
  const float* x;          // state positions (T = x > 0), or NULL when spins given
  const int8_t* spins;     // +1 selects; used when x == NULL
  const int32_t* blk_row;  // row range of each partial block [nblk + 1]
  int32_t nblk;
  int32_t n, R, G;
  double* partial;         // [nblk x R] scratch
  int64_t nnz = INT64_MAX; // CSR entries, where known (bounds-checked build)
};
cudaError_t launch_energy_partial(const Tiling& t, const EnergyArgs& a, cudaStream_t s);
// E[e*R + r] = sum of the event's block partials, in block order.
cudaError_t launch_energy_reduce(const double* partial, const int32_t* ev_blk0, int32_t E,
                                 int32_t R, double* E_out, cudaStream_t s);
// arg-min over replicas per event (ties -> lowest index).
cudaError_t launch_argmin(const double* E_all, int32_t E, int32_t R, double* best_E,
                          int32_t* best_r, cudaStream_t s);
cudaError_t launch_best_T(const float* x, const int32_t* row_event, const int32_t* best_r,
                          int32_t n, int32_t R, uint8_t* T, cudaStream_t s);

// ---------------------------------------------------------------- bSB adjoint
struct AdjArgs {
  const int32_t* rowptr;
  const int32_t* col;
  const void* J;             // FP32 or BF16, as the forward used
  const int8_t* cls;         // per nonzero: 1 = conflict
  const float* h;
  const double* quality;     // [n]
  const double* nconf;       // [n] conflicts per row
  int32_t n, R, G;
  float a0, c0, dt;
  const float* sched;        // a_k on the device (the forward's values)
  int32_t k;                 // the step being reversed
  const float* x;            // x_k (phase 2) or x_S (init)
  const float* ytil;         // y~_k
  const uint8_t* mask;       // m_k
  const float* frec;         // J x_k recorded by the forward recomputation
  float* lx;                 // adjoint of x
  float* ly;                 // adjoint of y
  float* lyt;                // adjoint of y~ (gathered by neighbours in phase 2)
  // phase 2 with the next step's phase 1 fused in: m_{k-1} and where the
  // adjoint of y~_{k-1} goes (not lyt, which neighbours still read); lx then
  // receives lx~_{k-1} and ly is not written. NULL mask_prev: plain phase 2.
  const uint8_t* mask_prev = nullptr;
  float* lyt_out = nullptr;
  double* gh;                // [n] dL/dh_i
  double* acc;               // [4]: loss, dL/ddt, dL/dc0, dL/dw_c (trajectory + explicit)
  double* ga;                // dL/da_k of this step (one double)
};
cudaError_t launch_adj_init(int jbf16, const Tiling& t, const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adj_phase1(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adj_phase2(int jbf16, const Tiling& t, const AdjArgs& a, cudaStream_t s);
// out[0] = sum_i gh_i (-quality_i / 2), out[1] = sum_i gh_i (-nconf_i / 4)
cudaError_t launch_adj_final(const AdjArgs& a, double* out, cudaStream_t s);


// ---------------------------------------------------------------- streamed step
// Warp-specialised step kernel (stream.cu). Rows are cut into blocks of
// kStreamBR rows; each block carries the sorted union of its rows' neighbour
// columns, padded to whole stages of kStreamSPS entries, with a kStreamBR-bit
// mask per entry telling which block rows use it. One producer warp per CTA
// copies the neighbour x rows (one replica tile of W replicas each) of that
// union into a shared-memory ring with bulk asynchronous copies; kStreamWarps
// consumer warps own kStreamRW rows each and accumulate every union entry
// their rows use, in ascending column order (the CSR order).
constexpr int kStreamWarps = 8;                       // consumer warps per CTA
constexpr int kStreamRW = 4;                          // rows per consumer warp
constexpr int kStreamBR = kStreamWarps * kStreamRW;   // rows per block (mask bits)
constexpr int kStreamSPS = 32;                        // union entries per ring stage
constexpr int kStreamThreads = (kStreamWarps + 1) * 32;

struct StreamArgs {
  const int32_t* rowptr;
  const void* J;             // float or __nv_bfloat16; the allocation is padded to 16 bytes
  const float* h;
  const int32_t* row_event;
  const float* c0_ev;
  const float* sched;
  int32_t k;
  float a0, dt, dta0;
  const float* xin;
  float* xout;
  float* y;
  int32_t n, R;
  const int32_t* cta_blk0;   // [grid + 1] first block of each CTA
  // [nblk + 1] per block: first row, first union entry (a multiple of
  // kStreamSPS), first J element of its 16-byte aligned J span, span bytes;
  // entry nblk = {n, total entries, 0, 0}
  const int4* blk;
  const int32_t* rjo;        // [n] rowptr[i] - first J element of the span of i's block
  const int32_t* ucol;       // union columns (padding entries: 0)
  const uint32_t* umask;     // bit q: block row q uses the column (padding entries: 0)
  int32_t grid;              // CTAs (one per SM)
  int32_t W;                 // replicas per tile: 256, 128 or 64
  int32_t tiles;             // R / W
  int32_t nst;               // ring stages
  int32_t jbuf_bytes;        // bytes of each of the two J staging buffers (multiple of 16)
  int* err;                  // set non-zero when a wait gives up (the kernel then returns)
  unsigned long long wait_ns;  // limit of every wait (globaltimer nanoseconds)
  // test hook: CTA 0's producer issues nothing for this stage (no arrival, no
  // copy), so the consumers' wait for it runs out; -1: off
  int32_t skip_stage;
};

// ---------------------------------------------------------------- factored step
// Coupling product split as jf * (M^T W M) x + residual x (factor.cu): group
// blocks g (e.g. one hit each) with K slots; U rows hold sum_{s'} W[s][s']
// T_{g,s'}, T_{g,s} the sum of x (dSB: of 2^-7 sgn) over the members of slot s.
struct FacSumArgs {
  const int32_t* gseg;   // [ng * K + 1] members of block g, slot s: gmem[gseg[gK+s] .. gseg[gK+s+1])
  const int32_t* gmem;   // member rows, ascending within a slot
  const int32_t* gout;   // [ng * K] U row written for (g, s); -1: not needed
  // work items: (block, first member, end member, scratch slot or -1); a block
  // of more than one chunk of members is split over several items, each adding
  // its chunk into a scratch slot, and the item that finishes last (counter
  // cnt[block]) sums the block's slots in chunk order and writes the U rows
  const int4* item;
  int32_t nitems;
  const int32_t* gnc;    // [ng] chunks of each block
  const int32_t* gscr0;  // [ng] first scratch slot of each block (-1: one chunk)
  int32_t* cnt;          // [ng x tiles] finished chunks per replica tile (zero between launches)
  float* scratch;        // [slots x K x R] chunk sums
  int32_t ng, K;
  uint32_t couple;       // bit 4 s + s': W[s][s'] = 1
  const float* xin;      // aSB / bSB: positions x_k [n x R]
  const uint8_t* sgn_in; // dSB: sign bytes of x_k [n x R]
  void* U;               // [U rows x R]: FP32 (aSB / bSB) or BF16 (dSB)
  int32_t R, G, NCH, tiles;
  int32_t n, urows;      // state rows and U rows (bounds-checked build)
};

// Row head of the factored step (fac_head_words() 32-bit words per row): the
// first kFacHead residual columns (0 past the row's end), the U rows
// (kFacHeadU words, -1 where none) and the first kFacHead residual values in
// the context precision. One line per row holds everything a row's first
// loads need, so they do not wait on the residual row pointer.
constexpr int kFacHead = 8, kFacHeadU = 4;
__host__ __device__ constexpr int fac_head_words(int jbytes) {
  return kFacHead + kFacHeadU + kFacHead * jbytes / 4;
}
struct FacHeadArgs {
  const int32_t* uidx;     // [n * K] U rows of each row (-1: none)
  const int32_t* rrowptr;  // residual CSR
  const int32_t* rcol;
  const void* rJ;
  uint32_t* head;          // [n * fac_head_words(jbytes)]
  int32_t n, K, jbytes;
};
cudaError_t launch_fac_head(const FacHeadArgs& a, cudaStream_t s);

struct FacStepArgs {
  const uint32_t* head;  // [n * fac_head_words(J bytes)] row heads
  int32_t K;
  float jf;              // factor weight in J units (-w / 4), exact in FP32
  const void* U;
  const int32_t* rrowptr;  // residual CSR [n + 1] (may hold the diagonal)
  const int32_t* rcol;
  const void* rJ;          // residual values, float or __nv_bfloat16 (exact)
  const float* h;
  const int32_t* row_event;
  const float* c0_ev;
  const float* sched;
  int32_t k;
  float a0, dt, dta0;
  const float* xin;
  float* xout;
  float* y;
  const uint8_t* sgn_in;   // dSB
  uint8_t* sgn_out;        // dSB
  int32_t n, R, G, NCH, tiles;
  int32_t urows;       // U rows (bounds-checked build)
  int64_t rnnz;        // residual entries (bounds-checked build)
};

// Lane-group shape of the factored kernels for R replicas (false: R not supported):
// G lanes per row, NCH 16-byte chunks per lane (aSB / bSB), tiles replica tiles.
bool fac_tiling(int variant, int R, int* G, int* NCH, int* tiles);
cudaError_t launch_fac_sum(int variant, const FacSumArgs& a, cudaStream_t s);
cudaError_t launch_step_fac(int variant, int jbf16, const FacStepArgs& a, cudaStream_t s);

// Replica-tile width of the streamed kernel for R replicas (0: not supported).
int stream_tile_width(int R);
// Dynamic shared memory of the streamed kernel for nst stages, or 0 when it
// does not fit; *nst_out receives the largest stage count that fits (<= 16).
size_t stream_smem(int W, int jbuf_bytes, int* nst_out);
cudaError_t launch_step_stream(int variant, int jbf16, const StreamArgs& a, size_t smem,
                               cudaStream_t s);
// Raise the dynamic shared-memory limit of every k_step_stream instance on the
// current device (call once per device before the first launch or capture).
cudaError_t stream_prepare();

// ---------------------------------------------------------------- row-group step
// k_step_rw (rw.cu): one warp owns a group of RW rows that share many
// neighbours and walks the sorted union of their columns; each union entry holds the column, an
// RW-bit mask of the group rows that use it and their J values (RW slots, 0
// where absent). A neighbour row of x is loaded once per group instead of once
// per row; every row still accumulates its nonzeros in CSR order, one FMA
// each, so states are identical to k_step's.
struct RwArgs {
  const int32_t* gptr;       // [ngroups + 1] first union entry of each row group
  const int32_t* grows;      // [ngroups x RW] rows of each group (-1: empty slot)
  const int32_t* ent;        // per entry: column << 4 | mask
  const void* ejv;           // per entry: RW J values (float or __nv_bfloat16)
  const float* h;
  const int32_t* row_event;
  const float* c0_ev;
  const float* sched;
  int32_t k;
  float a0, dt, dta0;
  const float* xin;
  float* xout;
  float* y;
  int32_t n, R;
  int32_t ngroups;
  int32_t gpc;               // row groups per CTA (a CTA walks a contiguous chunk)
  const uint8_t* sgn_in;     // dSB: sign bytes of x_k [n x R] gathered instead of x (NULL: use x)
  uint8_t* sgn_out;          // dSB: sign bytes of x_{k+1}, written with x_{k+1}
  // CTA b works on chunk cta_order[b] (chunks of gpc groups, heaviest first,
  // so that the last CTAs of a step are light); NULL: chunk b
  const int32_t* cta_order = nullptr;
  int32_t xrows = 0;         // rows of xin (state rows + U rows of the extended CSR; bounds-checked build)
};
constexpr int kRwMaxRows = 4;  // RW is 2 or 4 (the mask has 4 bits)
#ifndef SB_RW_BLOCK
#define SB_RW_BLOCK 128
#endif
constexpr int kRwBlock = SB_RW_BLOCK;  // threads per CTA of k_step_rw (one row group per warp)
// nch = 2: a warp covers 256 replicas of a row (two float4 per lane), grid.y = R / 256;
// nch = 1: 128 replicas, grid.y = R / 128. R must be a multiple of 128 * nch.
cudaError_t launch_step_rw(int variant, int jbf16, int rw, int nch, const RwArgs& a,
                           cudaStream_t s);
// ejv[i] = pos[i] >= 0 ? J[pos[i]] : 0 for i < count (J float or bf16 as jbf16 says)
cudaError_t launch_fill_ejv(const void* J, int jbf16, const int32_t* pos, int64_t count,
                            void* ejv, cudaStream_t s);

}  // namespace sbd
