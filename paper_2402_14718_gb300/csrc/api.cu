// C ABI of the SB solver: context life cycle, QUBO -> Ising set-up, SB runs
// (one launch per step, replayed from a captured CUDA graph), FP64 readout.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sb.h"
#include "device/kernels.cuh"
#include "device/probe.cuh"
#include "guard.h"

namespace sbh {
static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
}  // namespace sbh

using sbh::set_error;

namespace {

const int kEnergyRowsMin = 64;

// A run of steps is captured into a CUDA graph the second time the same run
// shape is asked for in a row, and replayed from then on; the first time it is
// launched directly, so a one-off run starts on the GPU without waiting for a
// capture and instantiation.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> key;   // run shape of exec
  std::vector<int64_t> seen;  // run shape last launched directly
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key.clear();
    seen.clear();
  }
};

// f(part, begin, end) over [0, count) cut into `parts` contiguous ranges, on up
// to `parts` host threads (fewer when the machine has fewer; sequential for
// small counts or when a thread cannot be started). Returns false if f threw
// (e.g. a failed allocation) in any part; the remaining parts still run.
template <typename F>
bool parallel_parts(int64_t count, int parts, F f, int64_t min_parallel = 8192) {
  std::atomic<bool> ok{true};
  auto run = [&](int p) {
    const int64_t b = count * p / parts, e = count * (p + 1) / parts;
    try {
      f(p, b, e);
    } catch (...) {
      ok = false;
    }
  };
  const unsigned hw = std::thread::hardware_concurrency();
  const int T = std::min(parts, (int)std::max(1u, std::min(hw, 16u)));
  if (T <= 1 || count < min_parallel) {
    for (int p = 0; p < parts; ++p) run(p);
    return ok;
  }
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int p; (p = next.fetch_add(1)) < parts;) run(p);
  };
  std::vector<std::thread> th;
  try {
    for (int t = 1; t < T; ++t) th.emplace_back(work);
  } catch (...) {
  }
  work();
  for (auto& x : th) x.join();
  return ok;
}

}  // namespace

struct sb_ctx {
  int device = 0;
  bool tiles_built = false;  // block tables of the tiled kernel are built on first use
  int32_t E = 1;
  int32_t n = 0;
  int64_t nnz = 0;
  int jbf16 = 0;
  std::vector<int32_t> ev_row0;  // [E + 1]
  std::vector<int64_t> ev_nnz;   // [E]
  std::vector<double> offset, sigma, c0_auto;
  // device: problem
  int32_t* d_rowptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_qval = nullptr;
  double* d_qlin = nullptr;
  void* d_J = nullptr;
  double* d_h64 = nullptr;
  float* d_h32 = nullptr;
  int32_t* d_row_event = nullptr;  // only when E > 1
  int32_t* d_ev_row0 = nullptr;
  double* d_offset = nullptr;
  double* d_sigma = nullptr;
  double* d_c0auto = nullptr;
  float* d_c0ev = nullptr;
  // device: state
  int32_t R = 0;
  float* d_x[2] = {nullptr, nullptr};
  float* d_y = nullptr;
  int cur = 0;
  bool have_state = false;
  float* d_sched = nullptr;  // default linear schedule
  int32_t sched_len = 0;
  double sched_a0 = 0.0;
  // readout (sized for eR replicas, independent of the state's R)
  int32_t eR = 0;
  int32_t energy_rows = 0, nblk = 0;
  int32_t* d_blk_row = nullptr;
  int32_t* d_ev_blk0 = nullptr;
  double* d_partial = nullptr;
  double* d_Eall = nullptr;
  double* d_bestE = nullptr;
  int32_t* d_bestr = nullptr;
  uint8_t* d_T = nullptr;
  int8_t* d_spins = nullptr;
  int32_t spins_cap_R = 0;
  // host copy of the (global) CSR structure, for weight updates and re-tiling
  std::vector<int32_t> h_rowptr, h_col;
  // class tags for the adjoint's weight-scale gradients (sb_set_weights)
  bool have_classes = false;
  int8_t* d_cls = nullptr;
  double* d_quality = nullptr;
  double* d_nconf = nullptr;
  // row-block tiling of the coupling product (k_step_tiled)
  bool tiled_ok = false;
  int32_t nb = 0;
  int32_t* d_blk_row0 = nullptr;
  int32_t* d_blk_u0 = nullptr;
  int32_t* d_ucol = nullptr;
  uint16_t* d_own = nullptr;
  void* d_tz = nullptr;
  // execution
  cudaStream_t cap_stream = nullptr;
  GraphCache graph;
  int use_graph = 1;
  int use_tiled = 0;
  int step_rt = 0;    // replica-tile width of the untiled kernel (0: automatic)
  int step_rpc = 0;   // rows per CTA of the untiled kernel (0: one row per group, -1: one wave)
  int step_unroll = 4;
  int dsb_signs = 1;  // dSB gathers int8 signs instead of FP32 positions
  // every |J_ij| < 2^118, so the sign-byte gathers may scale J by 2^7 exactly
  bool j_small = true;
  int groups = 1;     // replica groups run one after another (each for all steps)
  int l2_persist = 0; // mark each step's source x as L2-persisting (access-policy window)
  bool l2_raised = false;  // this context raised the persisting-L2 set-aside
  size_t l2_saved = 0;     // the set-aside before it did
  uint8_t* d_sgn[2] = {nullptr, nullptr};  // dSB sign bytes (0x3C, 0xBC, 0x00; signs.cuh)
  int sms = 0;
  // streamed step kernel (k_step_stream): per-CTA row chunks cut into blocks
  // with their neighbour-column unions; built on first use
  int use_stream = 0;
  bool stream_built = false;
  bool stream_ok = false;
  int32_t stream_grid = 0;
  int32_t stream_jbuf = 0;
  int32_t* d_s_cta = nullptr;
  int32_t* d_s_blk = nullptr;
  int32_t* d_s_rjo = nullptr;
  int32_t* d_s_ucol = nullptr;
  uint32_t* d_s_umask = nullptr;
  int* d_err = nullptr;  // set by a kernel whose bounded wait gave up
  unsigned long long wait_ns = 2000000000ull;  // limit of the streamed kernel's waits
  int32_t skip_stage = -1;  // test hook of the streamed kernel (SB_OPT_TEST_SKIP_STAGE)
  // row-group step kernel (k_step_rw): groups of RW rows and their union entries
  int rw_rows = -1;      // -1: automatic (2 for aSB / bSB, off for dSB); 0: off; 2 or 4
  // dispatch the row-group CTAs heaviest chunk first: 1 on, 0 off, -1 when
  // the gathered array fits in half of the L2 (otherwise row order keeps the
  // neighbour rows of CTAs in flight together in L2)
  int rw_heavy_first = -1;
  int r1_lanes = -1;  // one replica: lanes per row (0: one thread per row; -1: automatic)
  int l2_bytes = 0;
  int32_t* d_row_order = nullptr;  // chunk of each k_step_dsb16 CTA, heaviest first
  int32_t row_order_rpc = 0;
  int rw_built = 0;      // RW the tables below were built for (0: none)
  int32_t rw_ngroups = 0;
  int64_t rw_E = 0;
  int32_t* d_rw_gptr = nullptr;
  int32_t* d_rw_rows = nullptr;  // rows of each group (-1: empty slot)
  int32_t* d_rw_ent = nullptr;
  int32_t* d_rw_pos = nullptr;  // CSR position of each entry's RW slots (-1: absent)
  void* d_rw_ejv = nullptr;     // J of each entry's RW slots
  std::vector<int32_t> h_rw_gptr;  // host copy of the group pointers
  int32_t* d_rw_order = nullptr;   // chunk of each CTA, heaviest chunk first
  int32_t rw_order_gpc = 0;        // groups per chunk the order was made for
  // factored coupling product (sb_set_factor): group sums plus an exact residual
  bool fac_set = false;
  int fac_use = -1;          // SB_OPT_FACTOR: -1 or 1 use it when set and supported, 0 off
  int32_t fac_K = 0;
  uint32_t fac_couple = 0;   // bit 4 s + s': slots s and s' couple
  float fac_jf = 0.f;        // factor weight in J units (-w / 4)
  uint32_t fac_jf_bits = 0;  // the same in the context precision
  int32_t fac_ng = 0;        // group blocks with a U row in use
  int32_t fac_urows = 0;
  int32_t fac_rows = 0;      // rows in factored form
  int64_t fac_members = 0;   // member entries of those blocks
  int64_t fac_rnnz = 0;      // residual nonzeros
  int32_t fac_maxcount = 0;  // most members behind one U element
  int32_t* d_f_gseg = nullptr;
  int32_t* d_f_gmem = nullptr;
  int32_t* d_f_gout = nullptr;
  int4* d_f_item = nullptr;     // group-sum work items (block, member range, scratch slot)
  int4* d_f_item1 = nullptr;    // the same with one item per block (the dSB form)
  int32_t* d_f_gnc = nullptr;   // chunks per block
  int32_t* d_f_gscr0 = nullptr; // first scratch slot per block (-1: one chunk)
  int32_t fac_nitems = 0, fac_nslots = 0;
  int32_t* d_f_cnt = nullptr;   // finished chunks per (block, replica tile); zero between steps
  size_t f_cnt_count = 0;
  float* d_f_scr = nullptr;     // chunk sums [slots x K x R]
  size_t f_scr_count = 0;
  int32_t* d_f_uidx = nullptr;   // U rows of each row [n x K] (copied into the heads)
  uint32_t* d_f_head = nullptr;  // row heads of the factored step (sbd::fac_head_words per row)
  int32_t* d_f_rrowptr = nullptr;
  int32_t* d_f_rcol = nullptr;
  void* d_f_rJ = nullptr;
  void* d_f_U = nullptr;     // U rows of the current replica count
  size_t f_U_bytes = 0;
  // aSB / bSB with a factor: the row-group kernel over the extended CSR whose
  // columns n + u are the U rows (kept in the x buffers after the n state rows)
  std::vector<int32_t> h_fx_rowptr, h_fx_col;  // extended CSR structure
  void* d_f_xJ = nullptr;                      // its values (context precision)
  int frw_built = 0;                           // rows per warp of the tables below (0: none)
  int32_t frw_ngroups = 0;
  int64_t frw_E = 0;
  int32_t* d_frw_gptr = nullptr;
  int32_t* d_frw_rows = nullptr;
  int32_t* d_frw_ent = nullptr;
  int32_t* d_frw_pos = nullptr;
  void* d_frw_ejv = nullptr;
  int64_t x_rows = 0;                          // rows of each x buffer (>= n)
  // sb_backward's work memory, kept for the next call of the same shape
  struct AdjWork {
    int32_t n = 0, R = 0, S = 0, K = 0;
    float *ck_x = nullptr, *ck_y = nullptr, *seg_x = nullptr, *seg_yt = nullptr, *seg_f = nullptr;
    float *lx = nullptr, *ly = nullptr, *lyt[2] = {nullptr, nullptr};
    uint8_t* seg_m = nullptr;
    double *gh = nullptr, *acc = nullptr, *ga = nullptr;
  } adj;
};

namespace {

// On failure the error is reported and CUDA's last-error slot is cleared, so a
// non-sticky failure (e.g. an allocation) does not resurface at the next launch.
#define SB_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      cudaGetLastError();                                                          \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
      return e_ == cudaErrorMemoryAllocation ? SB_ERR_OOM : SB_ERR_CUDA;           \
    }                                                                              \
  } while (0)

template <typename T>
sb_status dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the non-sticky allocation error
    *p = nullptr;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return SB_ERR_OOM;
  }
  return SB_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

sb_status validate_csr(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                       const double* val, const double* lin, bool threads = true) {
  const int64_t min_par = threads ? 8192 : INT64_MAX;
  if (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz) {
    set_error("CSR: rowptr[0] must be 0 and rowptr[n] must equal nnz");
    return SB_ERR_CSR;
  }
  for (int32_t i = 0; i < n; ++i)  // every row range inside [0, nnz] before any col access
    if (rowptr[i + 1] < rowptr[i]) {
      set_error("CSR: rowptr decreases at row " + std::to_string(i));
      return SB_ERR_CSR;
    }
  // the first failing row (in row order) is reported; rows are checked in parallel parts
  struct Fail {
    int32_t row = INT32_MAX;
    sb_status st = SB_OK;
    std::string msg;
  };
  const int parts = 64;
  std::vector<Fail> fail(parts);
  auto first_failure = [&]() -> sb_status {
    const Fail* f = nullptr;
    for (const Fail& x : fail)
      if (x.st != SB_OK && (!f || x.row < f->row)) f = &x;
    if (!f) return SB_OK;
    set_error(f->msg);
    return f->st;
  };
  bool done = parallel_parts(n, parts, [&](int part, int64_t b, int64_t e) {
    Fail& F = fail[part];
    auto bad = [&](int32_t i, sb_status st, const std::string& m) {
      F.row = i;
      F.st = st;
      F.msg = m;
    };
    for (int32_t i = (int32_t)b; i < (int32_t)e && F.st == SB_OK; ++i) {
      if (!std::isfinite(lin[i])) {
        bad(i, SB_ERR_ARG, "linear term is not finite at row " + std::to_string(i));
        break;
      }
      for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int32_t j = col[p];
        if (j < 0 || j >= n) {
          bad(i, SB_ERR_CSR, "CSR: column out of range in row " + std::to_string(i));
          break;
        }
        if (j == i) {
          bad(i, SB_ERR_CSR, "CSR: diagonal entry in row " + std::to_string(i));
          break;
        }
        if (p > rowptr[i] && col[p - 1] >= j) {
          bad(i, SB_ERR_CSR, "CSR: columns not strictly ascending in row " + std::to_string(i));
          break;
        }
        if (!std::isfinite(val[p])) {
          bad(i, SB_ERR_ARG, "CSR: value not finite in row " + std::to_string(i));
          break;
        }
      }
    }
  }, min_par);
  sb_status st = first_failure();
  if (st) return st;
  if (!done) {
    set_error("CSR check: host allocation failed");
    return SB_ERR_OOM;
  }
  // symmetry: (i, j, v) needs (j, i, v)
  done = parallel_parts(n, parts, [&](int part, int64_t b, int64_t e) {
    Fail& F = fail[part];
    for (int32_t i = (int32_t)b; i < (int32_t)e && F.st == SB_OK; ++i)
      for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int32_t j = col[p];
        const int32_t* lo = col + rowptr[j];
        const int32_t* hi = col + rowptr[j + 1];
        const int32_t* f = std::lower_bound(lo, hi, i);
        if (f == hi || *f != i || val[rowptr[j] + (f - lo)] != val[p]) {
          F.row = i;
          F.st = SB_ERR_CSR;
          F.msg = "CSR: matrix is not symmetric at (" + std::to_string(i) + ", " +
                  std::to_string(j) + ")";
          break;
        }
      }
  }, min_par);
  st = first_failure();
  if (!st && !done) {
    set_error("CSR check: host allocation failed");
    return SB_ERR_OOM;
  }
  return st;
}

void free_readout(sb_ctx* c) {
  dfree(c->d_partial);
  dfree(c->d_Eall);
  c->eR = 0;
}

void free_state(sb_ctx* c) {
  dfree(c->d_x[0]);
  dfree(c->d_x[1]);
  c->x_rows = 0;
  dfree(c->d_y);
  dfree(c->d_sgn[0]);
  dfree(c->d_sgn[1]);
  c->R = 0;
  c->have_state = false;
  c->graph.reset();
}

void free_adj(sb_ctx* c) {
  sb_ctx::AdjWork& w = c->adj;
  dfree(w.ck_x);
  dfree(w.ck_y);
  dfree(w.seg_x);
  dfree(w.seg_yt);
  dfree(w.seg_f);
  dfree(w.seg_m);
  dfree(w.lx);
  dfree(w.ly);
  dfree(w.lyt[0]);
  dfree(w.lyt[1]);
  dfree(w.gh);
  dfree(w.acc);
  dfree(w.ga);
  w.n = w.R = w.S = w.K = 0;
}

void free_factor(sb_ctx* c) {
  dfree(c->d_f_gseg);
  dfree(c->d_f_gmem);
  dfree(c->d_f_gout);
  if (c->d_f_item) cudaFree(c->d_f_item);
  c->d_f_item = nullptr;
  if (c->d_f_item1) cudaFree(c->d_f_item1);
  c->d_f_item1 = nullptr;
  dfree(c->d_f_gnc);
  dfree(c->d_f_gscr0);
  dfree(c->d_f_cnt);
  dfree(c->d_f_scr);
  c->f_cnt_count = c->f_scr_count = 0;
  c->fac_nitems = c->fac_nslots = 0;
  dfree(c->d_f_uidx);
  if (c->d_f_head) cudaFree(c->d_f_head);
  c->d_f_head = nullptr;
  dfree(c->d_f_rrowptr);
  dfree(c->d_f_rcol);
  if (c->d_f_rJ) cudaFree(c->d_f_rJ);
  c->d_f_rJ = nullptr;
  if (c->d_f_U) cudaFree(c->d_f_U);
  c->d_f_U = nullptr;
  c->f_U_bytes = 0;
  if (c->d_f_xJ) cudaFree(c->d_f_xJ);
  c->d_f_xJ = nullptr;
  std::vector<int32_t>().swap(c->h_fx_rowptr);
  std::vector<int32_t>().swap(c->h_fx_col);
  dfree(c->d_frw_gptr);
  dfree(c->d_frw_rows);
  dfree(c->d_frw_ent);
  dfree(c->d_frw_pos);
  if (c->d_frw_ejv) cudaFree(c->d_frw_ejv);
  c->d_frw_ejv = nullptr;
  c->frw_built = 0;
  c->frw_ngroups = 0;
  c->frw_E = 0;
  c->fac_set = false;
  c->fac_K = c->fac_ng = c->fac_urows = c->fac_rows = c->fac_maxcount = 0;
  c->fac_members = c->fac_rnnz = 0;
  c->graph.reset();
}

void free_all(sb_ctx* c) {
  free_adj(c);
  free_factor(c);
  dfree(c->d_row_order);
  c->row_order_rpc = 0;
  free_state(c);
  free_readout(c);
  dfree(c->d_rowptr);
  dfree(c->d_col);
  dfree(c->d_qval);
  dfree(c->d_qlin);
  if (c->d_J) cudaFree(c->d_J);
  c->d_J = nullptr;
  dfree(c->d_h64);
  dfree(c->d_h32);
  dfree(c->d_row_event);
  dfree(c->d_ev_row0);
  dfree(c->d_offset);
  dfree(c->d_sigma);
  dfree(c->d_c0auto);
  dfree(c->d_c0ev);
  dfree(c->d_sched);
  dfree(c->d_blk_row);
  dfree(c->d_ev_blk0);
  dfree(c->d_bestE);
  dfree(c->d_bestr);
  dfree(c->d_T);
  dfree(c->d_spins);
  dfree(c->d_blk_row0);
  dfree(c->d_blk_u0);
  dfree(c->d_ucol);
  dfree(c->d_own);
  if (c->d_tz) cudaFree(c->d_tz);
  c->d_tz = nullptr;
  dfree(c->d_cls);
  dfree(c->d_quality);
  dfree(c->d_nconf);
  dfree(c->d_s_cta);
  dfree(c->d_s_blk);
  dfree(c->d_s_rjo);
  dfree(c->d_s_ucol);
  dfree(c->d_s_umask);
  dfree(c->d_err);
  dfree(c->d_rw_gptr);
  dfree(c->d_rw_rows);
  dfree(c->d_rw_ent);
  dfree(c->d_rw_pos);
  dfree(c->d_rw_order);
  c->rw_order_gpc = 0;
  if (c->d_rw_ejv) cudaFree(c->d_rw_ejv);
  c->d_rw_ejv = nullptr;
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
}

// (Re)build the energy block table: blocks of `rows` rows that never straddle an event.
sb_status ensure_energy_blocks(sb_ctx* c, int32_t rows) {
  if (c->energy_rows == rows && c->d_blk_row) return SB_OK;
  std::vector<int32_t> blk_row, ev_blk0;
  for (int32_t e = 0; e < c->E; ++e) {
    ev_blk0.push_back((int32_t)blk_row.size());
    for (int32_t r = c->ev_row0[e]; r < c->ev_row0[e + 1]; r += rows) blk_row.push_back(r);
  }
  ev_blk0.push_back((int32_t)blk_row.size());
  blk_row.push_back(c->n);
  dfree(c->d_blk_row);
  dfree(c->d_ev_blk0);
  sb_status st = dalloc(&c->d_blk_row, blk_row.size());
  if (st) return st;
  st = dalloc(&c->d_ev_blk0, ev_blk0.size());
  if (st) return st;
  SB_CUDA(cudaMemcpy(c->d_blk_row, blk_row.data(), blk_row.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_ev_blk0, ev_blk0.data(), ev_blk0.size() * 4, cudaMemcpyHostToDevice));
  c->nblk = (int32_t)blk_row.size() - 1;
  c->energy_rows = rows;
  return SB_OK;
}

sb_status ensure_state(sb_ctx* c, int32_t R) {
  if (c->R == R && c->d_y) return SB_OK;
  free_state(c);
  const size_t cnt = (size_t)c->n * R;
  // with a factor, the x buffers also hold the U rows after the n state rows
  const int64_t xr = (int64_t)c->n + (c->fac_set ? c->fac_urows : 0);
  sb_status st;
  if ((st = dalloc(&c->d_x[0], (size_t)xr * R)) || (st = dalloc(&c->d_x[1], (size_t)xr * R)) ||
      (st = dalloc(&c->d_y, cnt)))
    return st;
  c->x_rows = xr;
  c->R = R;
  c->cur = 0;
  c->have_state = false;
  return SB_OK;
}

sb_status ensure_readout(sb_ctx* c, int32_t R) {
  const sbd::Tiling t = sbd::make_tiling(R);
  const int32_t rows = std::max(kEnergyRowsMin, 256 / t.G);
  if (c->eR == R && c->energy_rows == rows && c->d_partial && c->d_Eall) return SB_OK;
  free_readout(c);
  sb_status st = ensure_energy_blocks(c, rows);
  if (st) return st;
  if ((st = dalloc(&c->d_partial, (size_t)c->nblk * R)) ||
      (st = dalloc(&c->d_Eall, (size_t)c->E * R)))
    return st;
  c->eR = R;
  return SB_OK;
}

// Cut rows into blocks (in row order) whose union of neighbour rows plus own
// rows stays within kTileUCap, nonzeros within kTileNzCap and rows within
// kTileRowCap; record each nonzero's index inside its block's sorted union.
struct TileHost {
  bool ok = true;
  std::vector<int32_t> row0, u0, ucol;
  std::vector<uint16_t> own, lidx;
};

TileHost build_tiles(int32_t n, const int32_t* rp, const int32_t* col) {
  TileHost t;
  t.own.assign(n, 0);
  t.lidx.assign((size_t)rp[n], 0);
  std::vector<int32_t> mark(n, -1), cur, sorted;
  int32_t row = 0;
  while (row < n) {
    const int32_t start = row;
    cur.clear();
    int64_t nz = 0;
    while (row < n && row - start < sbd::kTileRowCap) {
      int32_t add = mark[row] < 0 ? 1 : 0;
      for (int32_t p = rp[row]; p < rp[row + 1]; ++p) add += mark[col[p]] < 0 ? 1 : 0;
      const int64_t rnz = rp[row + 1] - rp[row];
      if ((int64_t)cur.size() + add > sbd::kTileUCap || nz + rnz > sbd::kTileNzCap) {
        if (row == start) {
          t.ok = false;
          return t;
        }
        break;
      }
      if (mark[row] < 0) {
        mark[row] = (int32_t)cur.size();
        cur.push_back(row);
      }
      for (int32_t p = rp[row]; p < rp[row + 1]; ++p)
        if (mark[col[p]] < 0) {
          mark[col[p]] = (int32_t)cur.size();
          cur.push_back(col[p]);
        }
      nz += rnz;
      ++row;
    }
    sorted = cur;
    std::sort(sorted.begin(), sorted.end());
    for (size_t k = 0; k < sorted.size(); ++k) mark[sorted[k]] = (int32_t)k;
    for (int32_t i = start; i < row; ++i) {
      t.own[i] = (uint16_t)mark[i];
      for (int32_t p = rp[i]; p < rp[i + 1]; ++p) t.lidx[p] = (uint16_t)mark[col[p]];
    }
    t.row0.push_back(start);
    t.u0.push_back((int32_t)t.ucol.size());
    t.ucol.insert(t.ucol.end(), sorted.begin(), sorted.end());
    for (int32_t v : cur) mark[v] = -1;
  }
  t.row0.push_back(n);
  t.u0.push_back((int32_t)t.ucol.size());
  return t;
}

sb_status setup_tiles(sb_ctx* c, const int32_t* rowptr, const int32_t* col) {
  TileHost t = build_tiles(c->n, rowptr, col);
  c->tiled_ok = false;
  if (!t.ok) return SB_OK;  // a row too long for a block: the generic kernel serves every run
  sb_status st;
  const size_t nnz = (size_t)c->nnz;
  uint16_t* d_lidx = nullptr;
  if ((st = dalloc(&c->d_blk_row0, t.row0.size())) || (st = dalloc(&c->d_blk_u0, t.u0.size())) ||
      (st = dalloc(&c->d_ucol, t.ucol.size())) || (st = dalloc(&c->d_own, (size_t)c->n)) ||
      (st = dalloc(&d_lidx, nnz)))
    return st;
  cudaError_t e = cudaMalloc(&c->d_tz, std::max<size_t>(nnz, 1) * (c->jbf16 ? 4 : 8));
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->d_tz = nullptr;
    dfree(d_lidx);
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return SB_ERR_OOM;
  }
  SB_CUDA(cudaMemcpy(c->d_blk_row0, t.row0.data(), t.row0.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_blk_u0, t.u0.data(), t.u0.size() * 4, cudaMemcpyHostToDevice));
  if (!t.ucol.empty())
    SB_CUDA(cudaMemcpy(c->d_ucol, t.ucol.data(), t.ucol.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_own, t.own.data(), (size_t)c->n * 2, cudaMemcpyHostToDevice));
  if (nnz) SB_CUDA(cudaMemcpy(d_lidx, t.lidx.data(), nnz * 2, cudaMemcpyHostToDevice));
  cudaError_t e1 = sbd::launch_pack_tz(c->d_J, c->jbf16, d_lidx, (int64_t)nnz, c->d_tz, 0);
  cudaError_t e2 = cudaDeviceSynchronize();
  dfree(d_lidx);
  SB_CUDA(e1);
  SB_CUDA(e2);
  c->nb = (int32_t)t.row0.size() - 1;
  c->tiled_ok = true;
  return SB_OK;
}

// Build the tiled kernel's block tables the first time the tiled kernel is wanted.
sb_status ensure_tiles(sb_ctx* c) {
  if (c->tiles_built) return SB_OK;
  sb_status st = setup_tiles(c, c->h_rowptr.data(), c->h_col.data());
  if (st) return st;
  c->tiles_built = true;
  return SB_OK;
}

// Tables of the streamed step kernel. Rows are split into `grid` contiguous
// chunks of about equal work (nonzeros + 8 per row), one per CTA; each chunk
// into blocks of kStreamBR rows. A block lists the sorted union of its rows'
// columns, one mask bit per block row that uses the column, padded with empty
// entries (column 0, mask 0) to a whole number (>= 1) of kStreamSPS-entry
// stages. jmax: the largest 16-byte aligned span of a block's J values.
struct StreamHost {
  bool ok = false;
  std::vector<int32_t> cta, row0, e0, ucol;
  std::vector<uint32_t> umask;
  std::vector<int32_t> blk;  // 4 per block (+ sentinel): row0, e0, first J element, J bytes
  std::vector<int32_t> rjo;  // [n] rowptr[i] - first J element of i's block
  int64_t jmax = 16;
};

StreamHost build_stream(int32_t n, const int32_t* rp, const int32_t* col, int grid, int esz) {
  StreamHost t;
  std::vector<int32_t> chunk(grid + 1, n);
  chunk[0] = 0;
  const long long total = (long long)rp[n] + 8LL * n;
  int32_t row = 0;
  long long acc = 0;
  for (int c = 1; c < grid; ++c) {
    const long long target = total * c / grid;
    while (row < n && acc + (rp[row + 1] - rp[row]) + 8 <= target) {
      acc += (rp[row + 1] - rp[row]) + 8;
      ++row;
    }
    chunk[c] = row;
  }
  std::vector<int32_t> mark(n, -1), uni;
  std::vector<uint32_t> mk;
  for (int c = 0; c < grid; ++c) {
    t.cta.push_back((int32_t)t.row0.size());
    for (int32_t r = chunk[c]; r < chunk[c + 1]; r += sbd::kStreamBR) {
      const int32_t r1 = std::min(r + sbd::kStreamBR, chunk[c + 1]);
      t.row0.push_back(r);
      t.e0.push_back((int32_t)t.ucol.size());
      uni.clear();
      for (int32_t i = r; i < r1; ++i)
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
          if (mark[col[p]] < 0) {
            mark[col[p]] = 0;
            uni.push_back(col[p]);
          }
      std::sort(uni.begin(), uni.end());
      for (size_t k = 0; k < uni.size(); ++k) mark[uni[k]] = (int32_t)k;
      mk.assign(uni.size(), 0u);
      for (int32_t i = r; i < r1; ++i)
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) mk[mark[col[p]]] |= 1u << (i - r);
      for (int32_t v : uni) mark[v] = -1;
      t.ucol.insert(t.ucol.end(), uni.begin(), uni.end());
      t.umask.insert(t.umask.end(), mk.begin(), mk.end());
      size_t pad = sbd::kStreamSPS - uni.size() % sbd::kStreamSPS;
      if (pad == (size_t)sbd::kStreamSPS && !uni.empty()) pad = 0;
      t.ucol.insert(t.ucol.end(), pad, 0);
      t.umask.insert(t.umask.end(), pad, 0u);
      const long long lo = ((long long)rp[r] * esz) & ~15LL;
      const long long hi = ((long long)rp[r1] * esz + 15) & ~15LL;
      t.jmax = std::max<int64_t>(t.jmax, hi - lo);
      if (t.ucol.size() > (size_t)INT32_MAX / 2) return t;
    }
  }
  t.cta.push_back((int32_t)t.row0.size());
  t.row0.push_back(n);
  t.e0.push_back((int32_t)t.ucol.size());
  // invariants the kernel relies on: every block has >= 1 whole stage, columns
  // are in range, and each row's mask bits count exactly its nonzeros
  const size_t nblk = t.row0.size() - 1;
  std::vector<int32_t> cnt(n, 0);
  for (size_t b = 0; b < nblk; ++b) {
    const int32_t e0 = t.e0[b], e1 = t.e0[b + 1];
    if (e1 <= e0 || (e1 - e0) % sbd::kStreamSPS || t.row0[b + 1] - t.row0[b] > sbd::kStreamBR ||
        t.row0[b + 1] <= t.row0[b])
      return t;
    for (int32_t e = e0; e < e1; ++e) {
      if (t.ucol[e] < 0 || t.ucol[e] >= n) return t;
      for (uint32_t m = t.umask[e]; m; m &= m - 1) {
        const int q = __builtin_ctz(m);
        if (t.row0[b] + q >= t.row0[b + 1]) return t;
        ++cnt[t.row0[b] + q];
      }
    }
  }
  for (int32_t i = 0; i < n; ++i)
    if (cnt[i] != rp[i + 1] - rp[i]) return t;
  t.rjo.assign(n, 0);
  for (size_t b = 0; b < nblk; ++b) {
    const int64_t lo = ((int64_t)rp[t.row0[b]] * esz) & ~int64_t(15);
    const int64_t hi = ((int64_t)rp[t.row0[b + 1]] * esz + 15) & ~int64_t(15);
    if (lo / esz > INT32_MAX) return t;
    t.blk.insert(t.blk.end(), {t.row0[b], t.e0[b], (int32_t)(lo / esz), (int32_t)(hi - lo)});
    for (int32_t i = t.row0[b]; i < t.row0[b + 1]; ++i) t.rjo[i] = rp[i] - (int32_t)(lo / esz);
  }
  t.blk.insert(t.blk.end(), {n, t.e0[nblk], 0, 0});
  t.ok = true;
  return t;
}

// Build the streamed kernel's tables the first time it is wanted (one CTA per SM).
sb_status ensure_stream(sb_ctx* c) {
  if (c->stream_built) return SB_OK;
  if (!c->sms) SB_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device));
  SB_CUDA(sbd::stream_prepare());
  StreamHost t = build_stream(c->n, c->h_rowptr.data(), c->h_col.data(), c->sms, c->jbf16 ? 2 : 4);
  c->stream_built = true;
  c->stream_ok = false;
  if (!t.ok) return SB_OK;  // the untiled kernel serves every run
  sb_status st;
  if ((st = dalloc(&c->d_s_cta, t.cta.size())) || (st = dalloc(&c->d_s_blk, t.blk.size())) ||
      (st = dalloc(&c->d_s_rjo, t.rjo.size())) || (st = dalloc(&c->d_s_ucol, t.ucol.size())) ||
      (st = dalloc(&c->d_s_umask, t.umask.size())))
    return st;
  SB_CUDA(cudaMemcpy(c->d_s_cta, t.cta.data(), t.cta.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_s_blk, t.blk.data(), t.blk.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_s_rjo, t.rjo.data(), t.rjo.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_s_ucol, t.ucol.data(), t.ucol.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_s_umask, t.umask.data(), t.umask.size() * 4, cudaMemcpyHostToDevice));
  c->stream_grid = c->sms;
  c->stream_jbuf = (int32_t)t.jmax;
  c->stream_ok = true;
  return SB_OK;
}

// Tables of the row-group kernel. Rows are cut into 64 contiguous parts (built
// on parallel host threads; the cut, and so the tables, do not depend on the
// thread count). Within a part, groups of RW rows are formed greedily in row
// order: the first row not yet placed anchors a group, which then takes, one
// at a time, the unplaced candidate of the same part (a neighbour of the
// anchor or one of the next 7 rows) adding the fewest new columns to the
// group's union. A group's entries are the sorted union of its rows' columns
// (a k-way merge of the CSR rows), each with an RW-bit mask and the CSR
// position of every slot. The grouping only decides which rows share loads;
// every row still accumulates its own nonzeros in CSR order.
struct RwHost {
  bool ok = false;
  std::vector<int32_t> gptr, rows, ent, pos;
};

RwHost build_rw(int32_t n, const int32_t* rp, const int32_t* col, int RW, int32_t ncols = -1) {
  RwHost t;
  if (ncols < 0) ncols = n;
  if (ncols >= (1 << 27) || RW < 2 || RW > sbd::kRwMaxRows) return t;
  const int parts = 64;
  struct Part {
    std::vector<int32_t> rows, cnt, ent, pos;
  };
  std::vector<Part> P(parts);
  const bool built = parallel_parts(n, parts, [&](int part, int64_t b64, int64_t e64) {
    const int32_t b = (int32_t)b64, e = (int32_t)e64;
    Part& q = P[part];
    if (e <= b) return;
    std::vector<char> placed((size_t)(e - b), 0);
    std::vector<int32_t> stamp((size_t)ncols, -1);
    int32_t ng = 0;
    if (RW == 2) {
      // The union entries of a pair are deg i + deg j - |N(i) & N(j)|, so the
      // pairing that reads the fewest rows is a maximum-weight matching with
      // the common-neighbour counts as weights. Greedy by decreasing weight over
      // the candidate pairs (neighbours within the part and the next seven
      // rows), ties by row order; zero-weight pairs last, so that rows still
      // share a warp. Groups follow in order of their first row.
      struct Cand {
        int32_t w, i, j;
      };
      std::vector<Cand> cands;
      for (int32_t i = b; i < e; ++i) {
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) stamp[col[p]] = i;
        auto add = [&](int32_t j) {
          int32_t w = 0;
          for (int32_t p = rp[j]; p < rp[j + 1]; ++p) w += stamp[col[p]] == i;
          cands.push_back({w, i, j});
        };
        // at most 192 neighbour candidates per row (the weights cost the sum of
        // the candidates' degrees; track QUBO rows have up to ~300 neighbours,
        // a dense QUBO could have thousands)
        int32_t taken = 0;
        for (int32_t p = rp[i]; p < rp[i + 1] && taken < 192; ++p)
          if (col[p] > i && col[p] < e) {
            add(col[p]);
            ++taken;
          }
        for (int32_t j = i + 1; j < std::min(e, i + 8); ++j)
          if (stamp[j] != i) add(j);  // not a neighbour: not added above
      }
      std::stable_sort(cands.begin(), cands.end(),
                       [](const Cand& x, const Cand& y) { return x.w > y.w; });
      std::vector<int32_t> mate((size_t)(e - b), -1);
      for (const Cand& c : cands)
        if (mate[c.i - b] < 0 && mate[c.j - b] < 0) {
          mate[c.i - b] = c.j;
          mate[c.j - b] = c.i;
        }
      for (int32_t i = b; i < e; ++i) {
        const int32_t m = mate[i - b];
        if (m >= 0 && m < i) continue;  // placed with its partner
        q.rows.push_back(i);
        q.rows.push_back(m);
        ++ng;
      }
    }
    for (int32_t i = b; i < e && RW != 2; ++i) {
      if (placed[i - b]) continue;
      placed[i - b] = 1;
      const size_t g0 = q.rows.size();
      q.rows.push_back(i);
      for (int32_t p = rp[i]; p < rp[i + 1]; ++p) stamp[col[p]] = ng;
      for (int k = 1; k < RW; ++k) {
        int32_t best = -1, best_add = INT32_MAX;
        auto consider = [&](int32_t j) {
          if (j < b || j >= e || placed[j - b]) return;
          int32_t add = 0;
          for (int32_t p = rp[j]; p < rp[j + 1] && add < best_add; ++p) add += stamp[col[p]] != ng;
          if (add < best_add) {
            best_add = add;
            best = j;
          }
        };
        for (int32_t p = rp[i]; p < rp[i + 1] && best_add > 0; ++p) consider(col[p]);
        for (int32_t j = i + 1; j < std::min(e, i + 8) && best_add > 0; ++j) consider(j);
        if (best < 0) break;
        placed[best - b] = 1;
        q.rows.push_back(best);
        for (int32_t p = rp[best]; p < rp[best + 1]; ++p) stamp[col[p]] = ng;
      }
      q.rows.resize(g0 + RW, -1);
      ++ng;
    }
    for (int32_t g = 0; g < ng; ++g) {
      int32_t p[sbd::kRwMaxRows], pe[sbd::kRwMaxRows];
      for (int k = 0; k < RW; ++k) {
        const int32_t row = q.rows[(size_t)g * RW + k];
        p[k] = row >= 0 ? rp[row] : 0;
        pe[k] = row >= 0 ? rp[row + 1] : 0;
      }
      const size_t before = q.ent.size();
      for (;;) {
        int32_t cmin = INT32_MAX;
        for (int k = 0; k < RW; ++k)
          if (p[k] < pe[k]) cmin = std::min(cmin, col[p[k]]);
        if (cmin == INT32_MAX) break;
        int32_t mask = 0;
        for (int k = 0; k < RW; ++k) {
          if (p[k] < pe[k] && col[p[k]] == cmin) {
            mask |= 1 << k;
            q.pos.push_back(p[k]++);
          } else {
            q.pos.push_back(-1);
          }
        }
        q.ent.push_back((cmin << 4) | mask);
      }
      q.cnt.push_back((int32_t)(q.ent.size() - before));
    }
  });
  if (!built) return t;  // a part ran out of host memory: no tables, the untiled kernel runs
  size_t E = 0, G = 0;
  for (const Part& q : P) {
    E += q.ent.size();
    G += q.cnt.size();
  }
  if (E > (size_t)INT32_MAX / 8) return t;
  t.gptr.reserve(G + 1);
  t.rows.reserve(G * RW);
  t.ent.reserve(E);
  t.pos.reserve(E * RW);
  t.gptr.push_back(0);
  for (const Part& q : P) {
    for (int32_t c : q.cnt) t.gptr.push_back(t.gptr.back() + c);
    t.rows.insert(t.rows.end(), q.rows.begin(), q.rows.end());
    t.ent.insert(t.ent.end(), q.ent.begin(), q.ent.end());
    t.pos.insert(t.pos.end(), q.pos.begin(), q.pos.end());
  }
  t.ok = true;
  return t;
}

// (Re)fill the entries' J slots from the current J (after create or a weight change).
sb_status refill_rw(sb_ctx* c) {
  if (!c->rw_built) return SB_OK;
  SB_CUDA(sbd::launch_fill_ejv(c->d_J, c->jbf16, c->d_rw_pos, c->rw_E * c->rw_built, c->d_rw_ejv,
                               0));
  SB_CUDA(cudaDeviceSynchronize());
  return SB_OK;
}

// Build the row-group tables for RW rows per warp the first time they are wanted.
sb_status ensure_rw(sb_ctx* c, int RW) {
  if (c->rw_built == RW) return SB_OK;
  RwHost t = build_rw(c->n, c->h_rowptr.data(), c->h_col.data(), RW);
  dfree(c->d_rw_gptr);
  dfree(c->d_rw_rows);
  dfree(c->d_rw_ent);
  dfree(c->d_rw_pos);
  dfree(c->d_rw_order);
  c->rw_order_gpc = 0;
  if (c->d_rw_ejv) cudaFree(c->d_rw_ejv);
  c->d_rw_ejv = nullptr;
  c->rw_built = 0;
  if (!t.ok) return SB_OK;  // the untiled kernel serves every run
  sb_status st;
  if ((st = dalloc(&c->d_rw_gptr, t.gptr.size())) || (st = dalloc(&c->d_rw_rows, t.rows.size())) ||
      (st = dalloc(&c->d_rw_ent, t.ent.size())) || (st = dalloc(&c->d_rw_pos, t.pos.size())))
    return st;
  {
    cudaError_t e = cudaMalloc(&c->d_rw_ejv, std::max<size_t>(t.pos.size(), 1) * (c->jbf16 ? 2 : 4));
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->d_rw_ejv = nullptr;
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return SB_ERR_OOM;
    }
  }
  SB_CUDA(cudaMemcpy(c->d_rw_gptr, t.gptr.data(), t.gptr.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_rw_rows, t.rows.data(), t.rows.size() * 4, cudaMemcpyHostToDevice));
  if (!t.ent.empty()) {
    SB_CUDA(cudaMemcpy(c->d_rw_ent, t.ent.data(), t.ent.size() * 4, cudaMemcpyHostToDevice));
    SB_CUDA(cudaMemcpy(c->d_rw_pos, t.pos.data(), t.pos.size() * 4, cudaMemcpyHostToDevice));
  }
  c->rw_ngroups = (int32_t)t.gptr.size() - 1;
  c->rw_E = (int64_t)t.ent.size();
  c->rw_built = RW;
  c->h_rw_gptr = std::move(t.gptr);
  return refill_rw(c);
}

// Dispatch order of the row-group CTAs: chunks of gpc consecutive groups
// sorted by decreasing cost (a CTA holds its slot until its slowest warp, so
// a chunk costs about its largest group: union entries plus a fixed share for
// the update), so that the CTAs that start last in a step are the light ones.
// Heavy-first dispatch pays where the end of a step is a large part of it (few
// waves of CTAs) and scattering the rows in flight costs nothing (the gathered
// array stays in L2); SB_OPT_HEAVY_FIRST forces it on or off.
bool heavy_first(sb_ctx* c, size_t gather_bytes, int64_t ctas) {
  if (c->rw_heavy_first >= 0) return c->rw_heavy_first > 0;
  if (!c->l2_bytes && cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, c->device))
    cudaGetLastError();
  if (!c->sms && cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device))
    cudaGetLastError();
  return gather_bytes * 2 <= (size_t)c->l2_bytes && ctas <= (int64_t)c->sms * 9 * 8;
}

// Dispatch order of the dSB sign-byte kernel's CTAs: chunks of rpc rows by
// decreasing cost (the largest row degree of the chunk plus a fixed share).
sb_status ensure_row_order(sb_ctx* c, int rpc) {
  if (c->d_row_order && c->row_order_rpc == rpc) return SB_OK;
  dfree(c->d_row_order);
  c->row_order_rpc = 0;
  const std::vector<int32_t>& rp = c->h_rowptr;
  const int32_t nch = (c->n + rpc - 1) / rpc;
  std::vector<int32_t> cost(nch, 0), order(nch);
  for (int32_t i = 0; i < c->n; ++i) {
    const int32_t w = rp[i + 1] - rp[i] + 8;
    int32_t& m = cost[i / rpc];
    if (w > m) m = w;
  }
  for (int32_t i = 0; i < nch; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
  sb_status st = dalloc(&c->d_row_order, order.size());
  if (st) return st;
  SB_CUDA(cudaMemcpy(c->d_row_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice));
  c->row_order_rpc = rpc;
  return SB_OK;
}

// One replica: lanes per row. Groups of lanes pay where rows alone leave the
// GPU's thread slots idle (they multiply the instructions of the coupling sum
// by the group width), so the automatic choice is the widest group with
// rows x lanes within the SMs' resident threads, else one thread per row.
int r1_lanes_for(sb_ctx* c) {
  if (c->r1_lanes >= 0) return c->r1_lanes;
  if (!c->sms && cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device))
    cudaGetLastError();
  const int64_t cap = (int64_t)std::max(c->sms, 1) * 2048;
  for (int G : {32, 16, 8})
    if ((int64_t)c->n * G <= cap) return G;
  return 0;
}

sb_status ensure_rw_order(sb_ctx* c, int gpc) {
  if (c->d_rw_order && c->rw_order_gpc == gpc) return SB_OK;
  dfree(c->d_rw_order);
  c->rw_order_gpc = 0;
  const std::vector<int32_t>& gp = c->h_rw_gptr;
  const int32_t G = (int32_t)gp.size() - 1;
  const int32_t nch = (G + gpc - 1) / gpc;
  std::vector<int32_t> cost(nch, 0), order(nch);
  for (int32_t g = 0; g < G; ++g) {
    const int32_t w = gp[g + 1] - gp[g] + 8;
    int32_t& m = cost[g / gpc];
    if (w > m) m = w;
  }
  for (int32_t i = 0; i < nch; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
  sb_status st = dalloc(&c->d_rw_order, order.size());
  if (st) return st;
  SB_CUDA(cudaMemcpy(c->d_rw_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice));
  c->rw_order_gpc = gpc;
  return SB_OK;
}

// The persisting-L2 set-aside belongs to the process's CUDA context. It is
// raised to the device maximum while a context marks x as persisting, and put
// back (with every persisting line returned to normal) when it stops, so that
// later runs get the whole L2.
sb_status l2_persist_on(sb_ctx* c) {
  if (c->l2_raised) return SB_OK;
  size_t old = 0;
  SB_CUDA(cudaDeviceGetLimit(&old, cudaLimitPersistingL2CacheSize));
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxPersistingL2CacheSize, c->device) == cudaSuccess &&
      v > 0)
    SB_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)v));
  c->l2_saved = old;
  c->l2_raised = true;
  return SB_OK;
}

sb_status l2_persist_off(sb_ctx* c) {
  if (!c->l2_raised) return SB_OK;
  SB_CUDA(cudaDeviceSynchronize());
  SB_CUDA(cudaCtxResetPersistingL2Cache());
  SB_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, c->l2_saved));
  c->l2_raised = false;
  return SB_OK;
}

// Report (and clear) the flag a kernel sets when one of its bounded waits gave up.
sb_status check_wait_flag(const sb_ctx* c) {
  int v = 0;
  SB_CUDA(cudaMemcpy(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) {
    SB_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
    set_error("a step kernel gave up waiting for its shared-memory pipeline (code " +
              std::to_string(v) + "); the state of that run is not valid");
    return SB_ERR_TIMEOUT;
  }
  return SB_OK;
}

// exactly representable in FP32 (and, with bf16, in BF16)
bool exact_in(double v, int bf16, uint32_t* bits) {
  const float f = (float)v;
  if ((double)f != v) return false;
  uint32_t u;
  memcpy(&u, &f, 4);
  if (bf16) {
    if (u & 0xffffu) return false;
    *bits = u >> 16;
  } else {
    *bits = u;
  }
  return true;
}

// |J_ij| <= sqrt(sum of J^2 over the event) = sigma_J sqrt(n (n - 1)) (the
// definition of sigma_J over the n (n - 1) off-diagonal places), so this bound
// keeps 2^7 J finite and exact in FP32 for the sign-byte gathers
void note_j_range(sb_ctx* c) {
  double m = 0.0;
  for (int32_t e = 0; e < c->E; ++e) {
    const double n = (double)(c->ev_row0[e + 1] - c->ev_row0[e]);
    if (n >= 2.0) m = std::max(m, c->sigma[e] * std::sqrt(n * (n - 1.0)));
  }
  c->j_small = m < 0x1p118;
}

sb_status create_common(sb_ctx* c, const int32_t* rowptr, const int32_t* col, const double* qval,
                        const double* qlin) {
  SB_CUDA(cudaGetDevice(&c->device));
  sb_status st;
  const size_t n = (size_t)c->n, nnz = (size_t)c->nnz;
  if ((st = dalloc(&c->d_rowptr, n + 1)) || (st = dalloc(&c->d_col, nnz)) ||
      (st = dalloc(&c->d_qval, nnz)) || (st = dalloc(&c->d_qlin, n)) ||
      (st = dalloc(&c->d_h64, n)) || (st = dalloc(&c->d_h32, n)) ||
      (st = dalloc(&c->d_ev_row0, (size_t)c->E + 1)) || (st = dalloc(&c->d_offset, c->E)) ||
      (st = dalloc(&c->d_sigma, c->E)) || (st = dalloc(&c->d_c0auto, c->E)) ||
      (st = dalloc(&c->d_c0ev, c->E)) || (st = dalloc(&c->d_bestE, c->E)) ||
      (st = dalloc(&c->d_bestr, c->E)) || (st = dalloc(&c->d_T, n)))
    return st;
  {
    // padded so that 16-byte aligned copies of any row range stay inside
    const size_t jb = ((std::max<size_t>(nnz, 1) * (c->jbf16 ? 2 : 4) + 15) & ~size_t(15)) + 16;
    cudaError_t e = cudaMalloc(&c->d_J, jb);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->d_J = nullptr;
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return SB_ERR_OOM;
    }
    SB_CUDA(cudaMemset(c->d_J, 0, jb));
  }
  if ((st = dalloc(&c->d_err, 1))) return st;
  SB_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
  SB_CUDA(cudaMemcpy(c->d_rowptr, rowptr, (n + 1) * 4, cudaMemcpyHostToDevice));
  if (nnz) {
    SB_CUDA(cudaMemcpy(c->d_col, col, nnz * 4, cudaMemcpyHostToDevice));
    SB_CUDA(cudaMemcpy(c->d_qval, qval, nnz * 8, cudaMemcpyHostToDevice));
  }
  SB_CUDA(cudaMemcpy(c->d_qlin, qlin, n * 8, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_ev_row0, c->ev_row0.data(), ((size_t)c->E + 1) * 4,
                     cudaMemcpyHostToDevice));
  if (c->E > 1) {
    std::vector<int32_t> re(n);
    for (int32_t e = 0; e < c->E; ++e)
      for (int32_t i = c->ev_row0[e]; i < c->ev_row0[e + 1]; ++i) re[i] = e;
    if ((st = dalloc(&c->d_row_event, n))) return st;
    SB_CUDA(cudaMemcpy(c->d_row_event, re.data(), n * 4, cudaMemcpyHostToDevice));
  }
  double *row_off = nullptr, *row_sq = nullptr;
  if ((st = dalloc(&row_off, n)) || (st = dalloc(&row_sq, n))) {
    dfree(row_off);
    dfree(row_sq);
    return st;
  }
  cudaError_t e1 = sbd::launch_convert(c->d_rowptr, c->d_col, c->d_qval, c->d_qlin, c->n, c->d_J,
                                       c->jbf16, c->d_h64, c->d_h32, row_off, row_sq, 0);
  cudaError_t e2 = sbd::launch_event_stats(row_off, row_sq, c->d_ev_row0, c->E, c->d_offset,
                                           c->d_sigma, c->d_c0auto, 0);
  cudaError_t e3 = cudaDeviceSynchronize();
  dfree(row_off);
  dfree(row_sq);
  SB_CUDA(e1);
  SB_CUDA(e2);
  SB_CUDA(e3);
  c->offset.resize(c->E);
  c->sigma.resize(c->E);
  c->c0_auto.resize(c->E);
  SB_CUDA(cudaMemcpy(c->offset.data(), c->d_offset, c->E * 8, cudaMemcpyDeviceToHost));
  SB_CUDA(cudaMemcpy(c->sigma.data(), c->d_sigma, c->E * 8, cudaMemcpyDeviceToHost));
  SB_CUDA(cudaMemcpy(c->c0_auto.data(), c->d_c0auto, c->E * 8, cudaMemcpyDeviceToHost));
  note_j_range(c);
  SB_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  return SB_OK;
}

// ---------------------------------------------------------------- factored coupling product
// J x = jf (M^T W M) x + Rs x with M the row -> (block, slot) incidence given by
// the caller, W the K x K slot-coupling pattern, jf = -w / 4, and the residual
// Rs = J - jf M^T W M formed here, exactly, from the context's J values
// (diagonal included; J_ii = 0). A row is kept in factored form when its residual is exactly
// representable in the context's J precision and its factored cost (U rows
// read + its share of the group sums + residual entries) is below its CSR
// length; other rows carry their plain CSR row as residual and read no U row.

sb_status set_factor(sb_ctx* c, int32_t n_ids, int32_t K, const int32_t* member,
                     const uint8_t* couple, double w) {
  const int32_t n = c->n;
  if (n_ids < 1 || K < 1 || K > 4 || !member || !couple || !std::isfinite(w) || w == 0.0) {
    set_error("sb_set_factor: need n_ids >= 1, 1 <= K <= 4, member, couple and a finite w != 0");
    return SB_ERR_ARG;
  }
  const double jf = -w / 4.0;
  uint32_t jf_bits;
  if (!exact_in(jf, c->jbf16, &jf_bits)) {
    set_error("sb_set_factor: -w / 4 must be exactly representable in the context's J precision");
    return SB_ERR_ARG;
  }
  uint32_t cm = 0;
  for (int s = 0; s < K; ++s)
    for (int s2 = 0; s2 < K; ++s2) {
      const uint8_t v = couple[s * K + s2];
      if (v > 1 || v != couple[s2 * K + s]) {
        set_error("sb_set_factor: couple must be a symmetric 0/1 matrix");
        return SB_ERR_ARG;
      }
      if (v) cm |= 1u << (4 * s + s2);
    }
  // members of each (id, slot), rows ascending (counting sort)
  const size_t nslot = (size_t)n_ids * K;
  std::vector<int64_t> seg(nslot + 1, 0);
  for (size_t t = 0; t < (size_t)n * K; ++t) {
    const int32_t g = member[t];
    if (g < -1 || g >= n_ids) {
      set_error("sb_set_factor: member ids must lie in [-1, n_ids)");
      return SB_ERR_ARG;
    }
    if (g >= 0) ++seg[(size_t)g * K + t % K + 1];
  }
  for (size_t t = 0; t < nslot; ++t) seg[t + 1] += seg[t];
  std::vector<int32_t> mem((size_t)seg[nslot]);
  {
    std::vector<int64_t> cur(seg.begin(), seg.end() - 1);
    for (int32_t i = 0; i < n; ++i)
      for (int s = 0; s < K; ++s) {
        const int32_t g = member[(size_t)i * K + s];
        if (g >= 0) mem[(size_t)cur[(size_t)g * K + s]++] = i;
      }
  }
  // the context's J values (the plain rows keep them; the residual is formed
  // from them, so a factored row uses the same couplings as its CSR row)
  const size_t nnz = (size_t)c->nnz, esz = c->jbf16 ? 2 : 4;
  std::vector<unsigned char> jraw(nnz * esz);
  if (nnz) SB_CUDA(cudaMemcpy(jraw.data(), c->d_J, nnz * esz, cudaMemcpyDeviceToHost));
  auto jval = [&](size_t t) -> double {
    uint32_t u = 0;
    memcpy(&u, jraw.data() + t * esz, esz);
    float f;
    u = esz == 2 ? u << 16 : u;
    memcpy(&f, &u, 4);
    return (double)f;
  };
  const int32_t* rp = c->h_rowptr.data();
  const int32_t* col = c->h_col.data();
  int32_t emax = 0;
  for (int32_t e = 0; e < c->E; ++e) emax = std::max(emax, c->ev_row0[e + 1] - c->ev_row0[e]);
  // rows in parallel parts: residual entries and the form of each row
  const int parts = 64;
  struct Part {
    std::vector<int32_t> rcol;
    std::vector<uint32_t> rbits;
    bool cross_event = false;
  };
  std::vector<Part> pt(parts);
  std::vector<int32_t> rcount(n);
  std::vector<uint8_t> isfac(n);
  const bool ok = parallel_parts(n, parts, [&](int p, int64_t b, int64_t e) {
    if (b >= e) return;
    Part& P = pt[p];
    // coupling counts m_ij of row i against the rows j of its event (dense,
    // zero between rows), the columns touched, and entries outside the CSR row
    std::vector<int32_t> cnt((size_t)emax, 0), touched, extra;
    std::vector<int32_t> rc;
    std::vector<uint32_t> rb;
    int32_t ev = (int32_t)(std::upper_bound(c->ev_row0.begin(), c->ev_row0.end(), (int32_t)b) -
                           c->ev_row0.begin()) - 1;
    for (int64_t i = b; i < e; ++i) {
      while (i >= c->ev_row0[ev + 1]) ++ev;
      const int32_t r0 = c->ev_row0[ev], r1 = c->ev_row0[ev + 1];
      touched.clear();
      int ns = 0;
      for (int s = 0; s < K; ++s) {
        const int32_t g = member[(size_t)i * K + s];
        if (g < 0) continue;
        ++ns;
        for (int s2 = 0; s2 < K; ++s2)
          if ((cm >> (4 * s + s2)) & 1u)
            for (int64_t t = seg[(size_t)g * K + s2]; t < seg[(size_t)g * K + s2 + 1]; ++t) {
              const int32_t j = mem[(size_t)t];
              if (j < r0 || j >= r1) {
                P.cross_event = true;
                continue;
              }
              if (cnt[(size_t)(j - r0)]++ == 0) touched.push_back(j);
            }
      }
      // residual J_ij - jf m_ij in column order: the CSR row merged with the
      // coupled rows outside it (the diagonal among them: J_ii = 0)
      rc.clear();
      rb.clear();
      bool exact = true;
      const int32_t q0 = rp[i], q1 = rp[i + 1];
      auto emit = [&](int32_t j, double r) {
        if (r == 0.0) return;
        uint32_t bits = 0;
        if (!exact_in(r, c->jbf16, &bits)) exact = false;
        rc.push_back(j);
        rb.push_back(bits);
      };
      for (int32_t q = q0; q < q1; ++q) {
        const int32_t j = col[q];
        int32_t& m = cnt[(size_t)(j - r0)];
        if (m > 0) m = -m;  // seen in the CSR row
      }
      extra.clear();
      for (int32_t j : touched)
        if (cnt[(size_t)(j - r0)] > 0) extra.push_back(j);
      std::sort(extra.begin(), extra.end());
      size_t xa = 0;
      for (int32_t q = q0; q < q1; ++q) {
        const int32_t j = col[q];
        for (; xa < extra.size() && extra[xa] < j; ++xa)
          emit(extra[xa], -jf * (double)cnt[(size_t)(extra[xa] - r0)]);
        const int32_t m = cnt[(size_t)(j - r0)];
        emit(j, jval((size_t)q) - jf * (double)(m < 0 ? -m : m));
      }
      for (; xa < extra.size(); ++xa) emit(extra[xa], -jf * (double)cnt[(size_t)(extra[xa] - r0)]);
      for (int32_t j : touched) cnt[(size_t)(j - r0)] = 0;
      for (int32_t q = q0; q < q1; ++q) cnt[(size_t)(col[q] - r0)] = 0;
      const int64_t fac_cost = 2 * (int64_t)ns + (int64_t)rc.size();
      if (ns > 0 && exact && fac_cost < (int64_t)(q1 - q0)) {
        isfac[i] = 1;
        rcount[i] = (int32_t)rc.size();
        P.rcol.insert(P.rcol.end(), rc.begin(), rc.end());
        P.rbits.insert(P.rbits.end(), rb.begin(), rb.end());
      } else {
        isfac[i] = 0;
        rcount[i] = q1 - q0;
        for (int32_t t = q0; t < q1; ++t) {
          uint32_t bits = 0;
          memcpy(&bits, jraw.data() + (size_t)t * esz, esz);
          P.rcol.push_back(col[t]);
          P.rbits.push_back(bits);
        }
      }
    }
  });
  if (!ok) {
    set_error("sb_set_factor: host allocation failed");
    return SB_ERR_OOM;
  }
  for (const Part& P : pt)
    if (P.cross_event) {
      set_error("sb_set_factor: a group id has members in more than one event");
      return SB_ERR_ARG;
    }
  std::vector<unsigned char>().swap(jraw);
  std::vector<int32_t> rrowptr((size_t)n + 1, 0);
  for (int32_t i = 0; i < n; ++i) {
    if ((int64_t)rrowptr[i] + rcount[i] > INT32_MAX) {
      set_error("sb_set_factor: residual too large");
      return SB_ERR_ARG;
    }
    rrowptr[i + 1] = rrowptr[i] + rcount[i];
  }
  const int64_t rnnz = rrowptr[n];
  // U rows read by factored rows, numbered in (id, slot) order
  std::vector<int32_t> urow(nslot, -1);
  for (int32_t i = 0; i < n; ++i)
    if (isfac[i])
      for (int s = 0; s < K; ++s) {
        const int32_t g = member[(size_t)i * K + s];
        if (g >= 0) urow[(size_t)g * K + s] = 0;
      }
  int64_t nu = 0;
  for (size_t t = 0; t < nslot; ++t)
    if (urow[t] == 0) urow[t] = (int32_t)nu++;
  if (nu > INT32_MAX) {
    set_error("sb_set_factor: too many U rows");
    return SB_ERR_ARG;
  }
  std::vector<int32_t> uidx((size_t)n * K, -1);
  int32_t nfac = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (!isfac[i]) continue;
    ++nfac;
    for (int s = 0; s < K; ++s) {
      const int32_t g = member[(size_t)i * K + s];
      if (g >= 0) uidx[(size_t)i * K + s] = urow[(size_t)g * K + s];
    }
  }
  // blocks with a U row in use: their members (all slots) and U outputs, by
  // event and, within an event, the blocks with most members first (a lane
  // group's time follows its block's size; the large blocks then start early,
  // not at the end)
  std::vector<int32_t> act;
  for (int32_t g = 0; g < n_ids; ++g) {
    bool used = false;
    for (int s = 0; s < K; ++s) used = used || urow[(size_t)g * K + s] >= 0;
    if (used) act.push_back(g);
  }
  {
    // stable counting sort by member count, descending
    std::vector<int64_t> sz(act.size());
    int64_t smax = 0;
    for (size_t t = 0; t < act.size(); ++t) {
      sz[t] = seg[(size_t)act[t] * K + K] - seg[(size_t)act[t] * K];
      smax = std::max(smax, sz[t]);
    }
    std::vector<int64_t> start((size_t)smax + 2, 0);
    for (int64_t v : sz) ++start[(size_t)(smax - v) + 1];
    for (size_t t = 0; t + 1 < start.size(); ++t) start[t + 1] += start[t];
    std::vector<int32_t> sorted(act.size());
    for (size_t t = 0; t < act.size(); ++t) sorted[(size_t)start[(size_t)(smax - sz[t])]++] = act[t];
    act.swap(sorted);
    // then, stably, by event: the blocks summed at the same time read the
    // sign bytes or x rows of a few events, which stay in L2 (sorted by size
    // over the whole batch they spread over every event's rows)
    if (c->E > 1) {
      std::vector<int32_t> bev(act.size());
      std::vector<int64_t> es((size_t)c->E + 1, 0);
      for (size_t t = 0; t < act.size(); ++t) {
        const int32_t g = act[t];
        int32_t row = 0;
        for (int s = 0; s < K; ++s)
          if (seg[(size_t)g * K + s + 1] > seg[(size_t)g * K + s]) {
            row = mem[(size_t)seg[(size_t)g * K + s]];
            break;
          }
        bev[t] = (int32_t)(std::upper_bound(c->ev_row0.begin(), c->ev_row0.end(), row) -
                           c->ev_row0.begin()) - 1;
        ++es[(size_t)bev[t] + 1];
      }
      for (size_t e = 0; e + 1 < es.size(); ++e) es[e + 1] += es[e];
      for (size_t t = 0; t < act.size(); ++t) sorted[(size_t)es[(size_t)bev[t]]++] = act[t];
      act.swap(sorted);
    }
  }
  int64_t total_mem = 0;
  for (int32_t g : act) total_mem += seg[(size_t)g * K + K] - seg[(size_t)g * K];
  if (total_mem > INT32_MAX) {
    set_error("sb_set_factor: too many member entries");
    return SB_ERR_ARG;
  }
  std::vector<int32_t> gseg(1, 0), gmem, gout;
  gseg.reserve(act.size() * K + 1);
  gout.reserve(act.size() * K);
  gmem.reserve((size_t)total_mem);
  int32_t maxcount = 0;
  for (int32_t g : act) {
    for (int s = 0; s < K; ++s) {
      const int64_t a0 = seg[(size_t)g * K + s], a1 = seg[(size_t)g * K + s + 1];
      gmem.insert(gmem.end(), mem.begin() + a0, mem.begin() + a1);
      gseg.push_back((int32_t)gmem.size());
      gout.push_back(urow[(size_t)g * K + s]);
      if (urow[(size_t)g * K + s] >= 0) {
        int64_t cnt = 0;
        for (int s2 = 0; s2 < K; ++s2)
          if ((cm >> (4 * s + s2)) & 1u) cnt += seg[(size_t)g * K + s2 + 1] - seg[(size_t)g * K + s2];
        maxcount = (int32_t)std::min<int64_t>(std::max<int64_t>(maxcount, cnt), INT32_MAX);
      }
    }
  }
  const int32_t ng = (int32_t)gout.size() / K;
  // work items of the group sums. aSB / bSB (one block per warp): blocks of
  // more than kChunk members are cut into near-equal chunks (a warp walks its
  // members one after another, so the largest block would otherwise set the
  // kernel's time). dSB (eight blocks per warp, advancing together): whole
  // blocks (measured faster there: the chunk sums' fences cost more than the
  // split saves).
  constexpr int64_t kChunk = 16;
  std::vector<int4> items, items1;
  items1.reserve((size_t)ng);
  for (int32_t ga = 0; ga < ng; ++ga)
    items1.push_back(make_int4(ga, gseg[(size_t)ga * K], gseg[(size_t)ga * K + K], -1));
  std::vector<int32_t> gnc(ng), gscr0(ng, -1);
  int32_t nslots = 0;
  for (int32_t ga = 0; ga < ng; ++ga) {
    const int64_t m0 = gseg[(size_t)ga * K], m1 = gseg[(size_t)ga * K + K], cnt = m1 - m0;
    const int32_t nc = (int32_t)std::max<int64_t>(1, (cnt + kChunk - 1) / kChunk);
    gnc[ga] = nc;
    if (nc == 1) {
      items.push_back(make_int4(ga, (int)m0, (int)m1, -1));
      continue;
    }
    gscr0[ga] = nslots;
    for (int32_t ci = 0; ci < nc; ++ci)
      items.push_back(make_int4(ga, (int)(m0 + ci * cnt / nc), (int)(m0 + (ci + 1) * cnt / nc),
                                nslots + ci));
    nslots += nc;
  }
  if ((int64_t)n + nu >= (1 << 27)) {
    set_error("sb_set_factor: rows plus U rows must stay below 2^27");
    return SB_ERR_ARG;
  }
  // the residual of all parts, in row order (each part copies its own range)
  std::vector<int32_t> rcol_all((size_t)rnnz);
  std::vector<unsigned char> rj_all((size_t)rnnz * esz);
  {
    std::vector<int64_t> pofs(parts + 1, 0);
    for (int p = 0; p < parts; ++p) pofs[p + 1] = pofs[p] + (int64_t)pt[p].rcol.size();
    parallel_parts(parts, parts, [&](int, int64_t b, int64_t e) {
      for (int64_t p = b; p < e; ++p) {
        Part& P = pt[(size_t)p];
        if (!P.rcol.empty())
          memcpy(rcol_all.data() + pofs[p], P.rcol.data(), P.rcol.size() * 4);
        unsigned char* d = rj_all.data() + (size_t)pofs[p] * esz;
        for (size_t t = 0; t < P.rbits.size(); ++t) memcpy(d + t * esz, &P.rbits[t], esz);  // low esz bytes (little-endian)
        std::vector<int32_t>().swap(P.rcol);
        std::vector<uint32_t>().swap(P.rbits);
      }
    }, 1);
  }
  // upload (replacing an earlier factor)
  SB_CUDA(cudaDeviceSynchronize());
  free_factor(c);
  sb_status st;
  if ((st = dalloc(&c->d_f_gseg, gseg.size())) || (st = dalloc(&c->d_f_gmem, std::max<size_t>(gmem.size(), 1))) ||
      (st = dalloc(&c->d_f_gout, std::max<size_t>(gout.size(), 1))) ||
      (st = dalloc(&c->d_f_uidx, uidx.size())) || (st = dalloc(&c->d_f_rrowptr, rrowptr.size())) ||
      (st = dalloc(&c->d_f_rcol, std::max<int64_t>(rnnz, 1)))) {
    free_factor(c);
    return st;
  }
  auto raw_alloc = [&](void** p, size_t bytes) -> sb_status {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      free_factor(c);
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return SB_ERR_OOM;
    }
    return SB_OK;
  };
  if ((st = raw_alloc(&c->d_f_rJ, std::max<int64_t>(rnnz, 1) * esz)) ||
      (st = raw_alloc(reinterpret_cast<void**>(&c->d_f_item), std::max<size_t>(items.size(), 1) * sizeof(int4))) ||
      (st = raw_alloc(reinterpret_cast<void**>(&c->d_f_item1), std::max<size_t>(items1.size(), 1) * sizeof(int4))) ||
      (st = raw_alloc(reinterpret_cast<void**>(&c->d_f_head),
                      std::max<size_t>((size_t)n * sbd::fac_head_words((int)esz) * 4, 16))))
    return st;
  if ((st = dalloc(&c->d_f_gnc, std::max<size_t>(gnc.size(), 1))) ||
      (st = dalloc(&c->d_f_gscr0, std::max<size_t>(gscr0.size(), 1)))) {
    free_factor(c);
    return st;
  }
  if (!items.empty())
    SB_CUDA(cudaMemcpy(c->d_f_item, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
  if (!items1.empty())
    SB_CUDA(cudaMemcpy(c->d_f_item1, items1.data(), items1.size() * sizeof(int4), cudaMemcpyHostToDevice));
  if (ng) {
    SB_CUDA(cudaMemcpy(c->d_f_gnc, gnc.data(), gnc.size() * 4, cudaMemcpyHostToDevice));
    SB_CUDA(cudaMemcpy(c->d_f_gscr0, gscr0.data(), gscr0.size() * 4, cudaMemcpyHostToDevice));
  }
  c->fac_nitems = (int32_t)items.size();
  c->fac_nslots = nslots;
  SB_CUDA(cudaMemcpy(c->d_f_gseg, gseg.data(), gseg.size() * 4, cudaMemcpyHostToDevice));
  if (!gmem.empty())
    SB_CUDA(cudaMemcpy(c->d_f_gmem, gmem.data(), gmem.size() * 4, cudaMemcpyHostToDevice));
  if (!gout.empty())
    SB_CUDA(cudaMemcpy(c->d_f_gout, gout.data(), gout.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_f_uidx, uidx.data(), uidx.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_f_rrowptr, rrowptr.data(), rrowptr.size() * 4, cudaMemcpyHostToDevice));
  if (rnnz) {
    SB_CUDA(cudaMemcpy(c->d_f_rcol, rcol_all.data(), (size_t)rnnz * 4, cudaMemcpyHostToDevice));
    SB_CUDA(cudaMemcpy(c->d_f_rJ, rj_all.data(), (size_t)rnnz * esz, cudaMemcpyHostToDevice));
  }
  {
    // row heads, formed on the device from the uploaded residual and U rows
    sbd::FacHeadArgs ha{};
    ha.uidx = c->d_f_uidx;
    ha.rrowptr = c->d_f_rrowptr;
    ha.rcol = c->d_f_rcol;
    ha.rJ = c->d_f_rJ;
    ha.head = c->d_f_head;
    ha.n = n;
    ha.K = K;
    ha.jbytes = (int)esz;
    SB_CUDA(sbd::launch_fac_head(ha, 0));
    SB_CUDA(cudaDeviceSynchronize());
  }
  c->fac_K = K;
  c->fac_couple = cm;
  c->fac_jf = (float)jf;
  c->fac_jf_bits = jf_bits;
  c->fac_ng = ng;
  c->fac_urows = (int32_t)nu;
  c->fac_rows = nfac;
  c->fac_members = (int64_t)gmem.size();
  c->fac_rnnz = rnnz;
  c->fac_maxcount = maxcount;
  c->fac_set = true;
  c->graph.reset();
  return SB_OK;
}

// The extended CSR of the row-group kernel (aSB / bSB with a factor): each
// row's residual, then its U rows as columns n + u (ascending) with the value
// jf. Formed on first use from the uploaded residual and U rows.
sb_status ensure_fx(sb_ctx* c) {
  if (c->d_f_xJ) return SB_OK;
  const int32_t n = c->n, K = c->fac_K;
  const size_t esz = c->jbf16 ? 2 : 4;
  const int64_t rnnz = c->fac_rnnz;
  std::vector<int32_t> rrowptr((size_t)n + 1), rcol((size_t)rnnz), uidx((size_t)n * K);
  std::vector<unsigned char> rj((size_t)rnnz * esz);
  SB_CUDA(cudaDeviceSynchronize());
  SB_CUDA(cudaMemcpy(rrowptr.data(), c->d_f_rrowptr, rrowptr.size() * 4, cudaMemcpyDeviceToHost));
  SB_CUDA(cudaMemcpy(uidx.data(), c->d_f_uidx, uidx.size() * 4, cudaMemcpyDeviceToHost));
  if (rnnz) {
    SB_CUDA(cudaMemcpy(rcol.data(), c->d_f_rcol, rcol.size() * 4, cudaMemcpyDeviceToHost));
    SB_CUDA(cudaMemcpy(rj.data(), c->d_f_rJ, rj.size(), cudaMemcpyDeviceToHost));
  }
  std::vector<int32_t> xrp((size_t)n + 1, 0);
  for (int32_t i = 0; i < n; ++i) {
    int64_t k = rrowptr[i + 1] - rrowptr[i];
    for (int s = 0; s < K; ++s) k += uidx[(size_t)i * K + s] >= 0 ? 1 : 0;
    if ((int64_t)xrp[i] + k > INT32_MAX) {
      set_error("sb_set_factor: extended CSR too large");
      return SB_ERR_ARG;
    }
    xrp[i + 1] = xrp[i] + (int32_t)k;
  }
  std::vector<int32_t> xcol((size_t)xrp[n]);
  std::vector<unsigned char> xj((size_t)xrp[n] * esz);
  for (int32_t i = 0; i < n; ++i) {
    int64_t dst = xrp[i];
    const int32_t r0 = rrowptr[i], r1 = rrowptr[i + 1];
    if (r1 > r0) {
      memcpy(xcol.data() + dst, rcol.data() + r0, (size_t)(r1 - r0) * 4);
      memcpy(xj.data() + (size_t)dst * esz, rj.data() + (size_t)r0 * esz, (size_t)(r1 - r0) * esz);
      dst += r1 - r0;
    }
    int32_t uu[4];
    int m = 0;
    for (int s = 0; s < K; ++s)
      if (uidx[(size_t)i * K + s] >= 0) uu[m++] = uidx[(size_t)i * K + s];
    std::sort(uu, uu + m);
    for (int t = 0; t < m; ++t, ++dst) {
      xcol[(size_t)dst] = n + uu[t];
      memcpy(xj.data() + (size_t)dst * esz, &c->fac_jf_bits, esz);
    }
  }
  cudaError_t e = cudaMalloc(&c->d_f_xJ, std::max<size_t>(xj.size(), 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->d_f_xJ = nullptr;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return SB_ERR_OOM;
  }
  if (!xj.empty()) SB_CUDA(cudaMemcpy(c->d_f_xJ, xj.data(), xj.size(), cudaMemcpyHostToDevice));
  c->h_fx_rowptr.swap(xrp);
  c->h_fx_col.swap(xcol);
  return SB_OK;
}

sb_status ensure_frw(sb_ctx* c, int RW) {
  if (c->frw_built == RW) return SB_OK;
  if (sb_status st0 = ensure_fx(c)) return st0;
  dfree(c->d_frw_gptr);
  dfree(c->d_frw_rows);
  dfree(c->d_frw_ent);
  dfree(c->d_frw_pos);
  if (c->d_frw_ejv) cudaFree(c->d_frw_ejv);
  c->d_frw_ejv = nullptr;
  c->frw_built = 0;
  RwHost t = build_rw(c->n, c->h_fx_rowptr.data(), c->h_fx_col.data(), RW, c->n + c->fac_urows);
  if (!t.ok) return SB_OK;  // the factored kernels serve the run instead
  sb_status st;
  if ((st = dalloc(&c->d_frw_gptr, t.gptr.size())) || (st = dalloc(&c->d_frw_rows, t.rows.size())) ||
      (st = dalloc(&c->d_frw_ent, std::max<size_t>(t.ent.size(), 1))) ||
      (st = dalloc(&c->d_frw_pos, std::max<size_t>(t.pos.size(), 1))))
    return st;
  {
    cudaError_t e = cudaMalloc(&c->d_frw_ejv, std::max<size_t>(t.pos.size(), 1) * (c->jbf16 ? 2 : 4));
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->d_frw_ejv = nullptr;
      set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return SB_ERR_OOM;
    }
  }
  SB_CUDA(cudaMemcpy(c->d_frw_gptr, t.gptr.data(), t.gptr.size() * 4, cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(c->d_frw_rows, t.rows.data(), t.rows.size() * 4, cudaMemcpyHostToDevice));
  if (!t.ent.empty()) {
    SB_CUDA(cudaMemcpy(c->d_frw_ent, t.ent.data(), t.ent.size() * 4, cudaMemcpyHostToDevice));
    SB_CUDA(cudaMemcpy(c->d_frw_pos, t.pos.data(), t.pos.size() * 4, cudaMemcpyHostToDevice));
  }
  c->frw_ngroups = (int32_t)t.gptr.size() - 1;
  c->frw_E = (int64_t)t.ent.size();
  SB_CUDA(sbd::launch_fill_ejv(c->d_f_xJ, c->jbf16, c->d_frw_pos, c->frw_E * RW, c->d_frw_ejv, 0));
  SB_CUDA(cudaDeviceSynchronize());
  c->frw_built = RW;
  return SB_OK;
}

// Grow both x buffers to `rows` rows of the current replica count, keeping
// the n state rows.
sb_status ensure_x_rows(sb_ctx* c, int64_t rows) {
  if (c->x_rows >= rows) return SB_OK;
  const size_t cnt = (size_t)rows * c->R, keep = (size_t)c->n * c->R;
  float* nx[2] = {nullptr, nullptr};
  sb_status st;
  if ((st = dalloc(&nx[0], cnt)) || (st = dalloc(&nx[1], cnt))) {
    dfree(nx[0]);
    dfree(nx[1]);
    return st;
  }
  SB_CUDA(cudaDeviceSynchronize());
  for (int k = 0; k < 2; ++k) {
    SB_CUDA(cudaMemcpy(nx[k], c->d_x[k], keep * 4, cudaMemcpyDeviceToDevice));
    dfree(c->d_x[k]);
    c->d_x[k] = nx[k];
  }
  c->x_rows = rows;
  c->graph.reset();
  return SB_OK;
}

sb_status check_run_args(sb_ctx* c, sb_variant variant, double a0, double c0, double dt,
                         int32_t steps) {
  if (!c) {
    set_error("null context");
    return SB_ERR_ARG;
  }
  if (variant < SB_ASB || variant > SB_DSB) {
    set_error("variant must be SB_ASB, SB_BSB or SB_DSB");
    return SB_ERR_ARG;
  }
  if (!(a0 > 0.0) || !std::isfinite(a0) || !(dt > 0.0) || !std::isfinite(dt) ||
      !std::isfinite(c0) || steps < 0) {
    set_error("a0 and dt must be positive and finite, c0 finite, steps >= 0");
    return SB_ERR_ARG;
  }
  return SB_OK;
}

// Enqueue `steps` SB steps reading x from c->d_x[c->cur]; flips c->cur.
sbd::Tiling step_tiling(const sb_ctx* c) {
  if (c->groups > 1 && c->R % (4 * c->groups) == 0) {
    const int rt = c->R / c->groups;
    if (rt <= 128 && ((rt / 4) & (rt / 4 - 1)) == 0) return sbd::make_tiling_rt(c->R, rt);
  }
  if (c->step_rt > 0 && c->R % c->step_rt == 0) return sbd::make_tiling_rt(c->R, c->step_rt);
  return sbd::make_tiling(c->R);
}

sb_status enqueue_steps(sb_ctx* c, int variant, double a0, double dt, int32_t steps,
                        const float* sched, cudaStream_t stream) {
  if (steps <= 0) return SB_OK;
  if (c->use_stream) {
    sb_status st0 = ensure_stream(c);
    if (st0) return st0;
  }
  if (c->use_tiled && c->R % sbd::kTileRT == 0) {
    sb_status st0 = ensure_tiles(c);
    if (st0) return st0;
  }
  // factored coupling product: set, not switched off, a supported replica count;
  // dSB needs the sign bytes and U sums that BF16 holds exactly
  int fG = 0, fNCH = 0, ftiles = 0;
  const int fac = (c->fac_set && c->fac_use != 0 && c->groups == 1 &&
                   sbd::fac_tiling(variant, c->R, &fG, &fNCH, &ftiles) &&
                   (variant != SB_DSB || (c->dsb_signs && c->j_small)))
                      ? 1 : 0;
  // dSB: BF16 U rows hold sums of at most 256 members exactly; larger blocks
  // take FP32 U rows (the dSB kernels' NCH = 2 instances)
  if (fac && variant == SB_DSB && c->fac_maxcount > 256) fNCH = 2;
  sbd::FacSumArgs fs{};
  sbd::FacStepArgs fa{};
  // aSB / bSB with R a multiple of 128: the row-group kernel over the extended
  // CSR, the U rows written into the x buffer after the n state rows
  int frw = 0;
  if (fac && variant != SB_DSB && c->R % 128 == 0 && c->rw_rows != 0 && c->step_rt == 0) {
    sb_status st0 = ensure_frw(c, 2);
    if (st0) return st0;
    if (c->frw_built == 2) {
      if ((st0 = ensure_x_rows(c, (int64_t)c->n + c->fac_urows))) return st0;
      frw = 1;
    }
  }
  if (fac && !frw) {
    const size_t ub = (size_t)std::max(c->fac_urows, 1) * c->R * (variant == SB_DSB && fNCH == 1 ? 2 : 4);
    if (ub > c->f_U_bytes) {
      if (c->d_f_U) cudaFree(c->d_f_U);
      c->d_f_U = nullptr;
      c->f_U_bytes = 0;
      cudaError_t e = cudaMalloc(&c->d_f_U, ub);
      if (e != cudaSuccess) {
        cudaGetLastError();
        c->d_f_U = nullptr;
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return SB_ERR_OOM;
      }
      c->f_U_bytes = ub;
      c->graph.reset();
    }
  }
  if (fac) {
    // chunk counters (zeroed once: every launch leaves them at zero) and chunk sums
    const size_t cnt_need = (size_t)std::max(c->fac_ng, 1) * ftiles;
    if (cnt_need > c->f_cnt_count) {
      dfree(c->d_f_cnt);
      c->f_cnt_count = 0;
      sb_status st0 = dalloc(&c->d_f_cnt, cnt_need);
      if (st0) return st0;
      SB_CUDA(cudaMemset(c->d_f_cnt, 0, cnt_need * 4));
      c->f_cnt_count = cnt_need;
      c->graph.reset();
    }
    const size_t scr_need = (size_t)std::max(c->fac_nslots, 1) * c->fac_K * c->R;
    if (scr_need > c->f_scr_count) {
      dfree(c->d_f_scr);
      c->f_scr_count = 0;
      sb_status st0 = dalloc(&c->d_f_scr, scr_need);
      if (st0) return st0;
      c->f_scr_count = scr_need;
      c->graph.reset();
    }
    fs.item = variant == SB_DSB ? c->d_f_item1 : c->d_f_item;
    fs.nitems = variant == SB_DSB ? c->fac_ng : c->fac_nitems;
    fs.gnc = c->d_f_gnc;
    fs.gscr0 = c->d_f_gscr0;
    fs.cnt = c->d_f_cnt;
    fs.scratch = c->d_f_scr;
    fs.gseg = c->d_f_gseg;
    fs.gmem = c->d_f_gmem;
    fs.gout = c->d_f_gout;
    fs.ng = c->fac_ng;
    fs.K = c->fac_K;
    fs.couple = c->fac_couple;
    fs.U = c->d_f_U;
    fs.R = c->R;
    fs.G = fG;
    fs.NCH = fNCH;
    fs.tiles = ftiles;
    fs.n = c->n;
    fs.urows = c->fac_urows;
    fa.urows = c->fac_urows;
    fa.rnnz = c->fac_rnnz;
    fa.head = c->d_f_head;
    fa.K = c->fac_K;
    fa.jf = c->fac_jf;
    fa.U = c->d_f_U;
    fa.rrowptr = c->d_f_rrowptr;
    fa.rcol = c->d_f_rcol;
    fa.rJ = c->d_f_rJ;
    fa.h = c->d_h32;
    fa.row_event = c->d_row_event;
    fa.c0_ev = c->d_c0ev;
    fa.sched = sched;
    fa.a0 = (float)a0;
    fa.dt = (float)dt;
    fa.dta0 = (float)(dt * a0);
    fa.y = c->d_y;
    fa.n = c->n;
    fa.R = c->R;
    fa.G = fG;
    fa.NCH = fNCH;
    fa.tiles = ftiles;
  }
  // streamed kernel: chosen, tables valid, a supported replica count, and a ring that fits
  sbd::StreamArgs sa{};
  size_t s_smem = 0;
  if (!fac && c->use_stream && c->stream_ok && c->groups == 1) {
    sa.W = sbd::stream_tile_width(c->R);
    if (sa.W) s_smem = sbd::stream_smem(sa.W, c->stream_jbuf, &sa.nst);
  }
  const int streamed = s_smem ? 1 : 0;
  // row-group kernel: chosen, R a multiple of 128, tables valid
  int rw = 0, rw_nch = 0;
  sbd::RwArgs ra{};
  // automatic choice: row groups of 2 for aSB / bSB, which gather FP32 x;
  // dSB keeps its sign-byte kernel (fewer instructions per neighbour)
  const int rw_want = c->rw_rows < 0 ? (variant == SB_DSB ? 0 : 2) : c->rw_rows;
  const bool rw_auto_ok = c->rw_rows >= 0 || (!c->use_tiled && c->step_rt == 0);
  if (!fac && !streamed && rw_want && rw_auto_ok && c->groups == 1 && c->R % 128 == 0) {
    sb_status st0 = ensure_rw(c, rw_want);
    if (st0) return st0;
    if (c->rw_built == rw_want) {
      rw = rw_want;
      rw_nch = (c->R % 256 == 0 && c->step_rt != 128) ? 2 : 1;
      ra.gptr = c->d_rw_gptr;
      ra.grows = c->d_rw_rows;
      ra.ent = c->d_rw_ent;
      ra.ejv = c->d_rw_ejv;
      ra.h = c->d_h32;
      ra.row_event = c->d_row_event;
      ra.c0_ev = c->d_c0ev;
      ra.sched = sched;
      ra.a0 = (float)a0;
      ra.dt = (float)dt;
      ra.dta0 = (float)(dt * a0);
      ra.y = c->d_y;
      ra.n = c->n;
      ra.R = c->R;
      ra.ngroups = c->rw_ngroups;
      ra.gpc = std::max(sbd::kRwBlock / 32, c->step_rpc > 0 ? c->step_rpc / rw : 0);
      ra.cta_order = nullptr;
      const bool sgn_rw = variant == SB_DSB && c->dsb_signs && c->j_small;
      const int64_t ctas = ((int64_t)c->rw_ngroups + ra.gpc - 1) / ra.gpc;
      if (heavy_first(c, (size_t)c->n * c->R * (sgn_rw ? 1 : 4), ctas)) {
        st0 = ensure_rw_order(c, ra.gpc);
        if (st0) return st0;
        ra.cta_order = c->d_rw_order;
      }
    }
  }
  if (frw) {
    rw = 2;
    rw_nch = c->R % 256 == 0 ? 2 : 1;
    ra.gptr = c->d_frw_gptr;
    ra.grows = c->d_frw_rows;
    ra.ent = c->d_frw_ent;
    ra.ejv = c->d_frw_ejv;
    ra.h = c->d_h32;
    ra.row_event = c->d_row_event;
    ra.c0_ev = c->d_c0ev;
    ra.sched = sched;
    ra.a0 = (float)a0;
    ra.dt = (float)dt;
    ra.dta0 = (float)(dt * a0);
    ra.y = c->d_y;
    ra.n = c->n;
    ra.R = c->R;
    ra.xrows = c->n + c->fac_urows;  // the extended CSR's columns n + u are U rows
    ra.ngroups = c->frw_ngroups;
    ra.gpc = std::max(sbd::kRwBlock / 32, c->step_rpc > 0 ? c->step_rpc / 2 : 0);
    ra.cta_order = nullptr;
    ra.sgn_in = nullptr;
    ra.sgn_out = nullptr;
  }
  if (streamed) {
    sa.rowptr = c->d_rowptr;
    sa.J = c->d_J;
    sa.h = c->d_h32;
    sa.row_event = c->d_row_event;
    sa.c0_ev = c->d_c0ev;
    sa.sched = sched;
    sa.a0 = (float)a0;
    sa.dt = (float)dt;
    sa.dta0 = (float)(dt * a0);
    sa.y = c->d_y;
    sa.n = c->n;
    sa.R = c->R;
    sa.cta_blk0 = c->d_s_cta;
    sa.blk = reinterpret_cast<const int4*>(c->d_s_blk);
    sa.rjo = c->d_s_rjo;
    sa.ucol = c->d_s_ucol;
    sa.umask = c->d_s_umask;
    sa.grid = c->stream_grid;
    sa.tiles = c->R / sa.W;
    sa.jbuf_bytes = c->stream_jbuf;
    sa.err = c->d_err;
    sa.wait_ns = c->wait_ns;
    sa.skip_stage = c->skip_stage;
  }
  // the 16-replica dSB kernel exists only with sign bytes: its tiling and the
  // byte condition below must agree
  const bool dsb16 = !fac && !streamed && !rw && variant == SB_DSB && c->dsb_signs && c->j_small &&
                     c->step_rt == 0 &&
                     c->groups == 1 && sbd::dsb16_ok(c->R) &&
                     !(c->tiled_ok && c->use_tiled && c->R % sbd::kTileRT == 0);
  const sbd::Tiling t = dsb16 ? sbd::make_tiling_dsb16(c->R) : step_tiling(c);
  sbd::StepArgs a;
  a.rowptr = c->d_rowptr;
  a.col = c->d_col;
  a.J = c->d_J;
  a.h = c->d_h32;
  a.row_event = c->d_row_event;
  a.c0_ev = c->d_c0ev;
  a.sched = sched;
  a.a0 = (float)a0;
  a.dt = (float)dt;
  a.dta0 = (float)(dt * a0);
  a.y = c->d_y;
  a.n = c->n;
  a.R = c->R;
  a.G = t.G;
  a.unroll = c->step_unroll;
  a.tile0 = 0;
  a.nnz = c->nnz;
  a.rpc = std::max(256 / t.G, c->step_rpc);
  a.frec = nullptr;
  if (c->step_rpc < 0) {  // one wave: every resident CTA walks one contiguous row chunk
    if (!c->sms) SB_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device));
    const long long slots =
        (long long)c->sms * sbd::step_blocks_per_sm(variant, c->jbf16, t, a.unroll);
    const long long per = ((long long)c->n * t.tiles + slots - 1) / slots;
    a.rpc = (int)std::max<long long>(256 / t.G, per);
  }
  a.ytil = nullptr;
  a.mask = nullptr;
  a.sgn_in = nullptr;
  a.sgn_out = nullptr;
  a.cta_order = nullptr;
  a.r1_lanes = r1_lanes_for(c);
  if (dsb16) {
    const int rpc16 = sbd::dsb16_rows_per_cta(a.rpc);
    if (heavy_first(c, (size_t)c->n * c->R, ((int64_t)c->n + rpc16 - 1) / rpc16)) {
      sb_status st2 = ensure_row_order(c, rpc16);
      if (st2) return st2;
      a.cta_order = c->d_row_order;
    }
  }
  const int tiled =
      (!fac && !streamed && !rw && c->tiled_ok && c->use_tiled && c->R % sbd::kTileRT == 0) ? 1 : 0;
  sbd::TiledArgs ta;
  ta.blk_row0 = c->d_blk_row0;
  ta.blk_u0 = c->d_blk_u0;
  ta.ucol = c->d_ucol;
  ta.own = c->d_own;
  ta.rowptr = c->d_rowptr;
  ta.tz = c->d_tz;
  ta.h = c->d_h32;
  ta.row_event = c->d_row_event;
  ta.c0_ev = c->d_c0ev;
  ta.sched = sched;
  ta.a0 = a.a0;
  ta.dt = a.dt;
  ta.dta0 = a.dta0;
  ta.y = c->d_y;
  ta.n = c->n;
  ta.R = c->R;
  ta.nb = c->nb;
  const int sgn = (variant == SB_DSB && c->dsb_signs && c->j_small && !tiled && !streamed &&
                   c->R % 4 == 0) ? 1 : 0;
  if (sgn && !(c->d_sgn[0] && c->d_sgn[1])) {
    dfree(c->d_sgn[0]);  // a failed earlier attempt may have left one of the pair
    dfree(c->d_sgn[1]);
    sb_status st2;
    const size_t cnt = (size_t)c->n * c->R;
    if ((st2 = dalloc(&c->d_sgn[0], cnt)) || (st2 = dalloc(&c->d_sgn[1], cnt))) return st2;
  }

  size_t win_max = 0;
  if (c->l2_persist) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxAccessPolicyWindowSize, c->device) == cudaSuccess)
      win_max = (size_t)v;
  }
  auto set_window = [&](const void* base, cudaStream_t st) -> cudaError_t {
    if (!c->l2_persist || !win_max) return cudaSuccess;
    cudaStreamAttrValue v = {};
    v.accessPolicyWindow.base_ptr = const_cast<void*>(base);
    v.accessPolicyWindow.num_bytes = std::min(win_max, (size_t)c->n * c->R * sizeof(float));
    v.accessPolicyWindow.hitRatio = 1.0f;
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    return cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v);
  };
  const int ngroups =
      (!fac && !streamed && !rw && !tiled && !dsb16 && c->groups > 1 && t.tiles == c->groups) ? c->groups : 1;
  // factored dSB with sign bytes: neighbours read only the sign bytes
  // (ping-pong), so each row updates its own x in place and the kernel skips
  // writing back values that did not change; the other paths ping-pong x
  const bool x_inplace = fac && sgn && ngroups == 1;
  auto launch = [&](int32_t k, int cur, cudaStream_t st) -> cudaError_t {
    float* const xi = x_inplace ? c->d_x[c->cur] : c->d_x[cur];
    float* const xo = x_inplace ? xi : c->d_x[cur ^ 1];
    cudaError_t ew = set_window(xi, st);
    if (ew != cudaSuccess) return ew;
    if (sgn) {
      a.sgn_in = c->d_sgn[cur];
      a.sgn_out = c->d_sgn[cur ^ 1];
    }
    if (fac) {
      fs.xin = xi;
      fs.sgn_in = sgn ? c->d_sgn[cur] : nullptr;
      if (frw) fs.U = c->d_x[cur] + (size_t)c->n * c->R;
      cudaError_t ef = sbd::launch_fac_sum(variant, fs, st);
      if (ef != cudaSuccess || frw) {
        if (ef != cudaSuccess) return ef;
        ra.k = k;
        ra.xin = c->d_x[cur];
        ra.xout = c->d_x[cur ^ 1];
        return sbd::launch_step_rw(variant, c->jbf16, 2, rw_nch, ra, st);
      }
      fa.k = k;
      fa.xin = xi;
      fa.xout = xo;
      fa.sgn_in = sgn ? c->d_sgn[cur] : nullptr;
      fa.sgn_out = sgn ? c->d_sgn[cur ^ 1] : nullptr;
      return sbd::launch_step_fac(variant, c->jbf16, fa, st);
    }
    if (streamed) {
      sa.k = k;
      sa.xin = c->d_x[cur];
      sa.xout = c->d_x[cur ^ 1];
      return sbd::launch_step_stream(variant, c->jbf16, sa, s_smem, st);
    }
    if (rw) {
      ra.k = k;
      ra.xin = xi;
      ra.xout = xo;
      ra.sgn_in = sgn ? c->d_sgn[cur] : nullptr;
      ra.sgn_out = sgn ? c->d_sgn[cur ^ 1] : nullptr;
      return sbd::launch_step_rw(variant, c->jbf16, rw, rw_nch, ra, st);
    }
    if (tiled) {
      ta.k = k;
      ta.xin = c->d_x[cur];
      ta.xout = c->d_x[cur ^ 1];
      return sbd::launch_step_tiled(variant, c->jbf16, ta, st);
    }
    a.k = k;
    a.xin = xi;
    a.xout = xo;
    return sbd::launch_step(variant, c->jbf16, t, a, st);
  };
  const size_t NR = (size_t)c->n * c->R;
  sbd::Tiling tg = t;
  if (ngroups > 1) tg.tiles = 1;
  // all steps for replica group g (tiles g), then the next group: each group's
  // working set stays in L2 for the whole run; parity ends the same for all
  auto launch_all = [&](int cur0, cudaStream_t st) -> cudaError_t {
    cudaError_t err = cudaSuccess;
    if (sgn) err = sbd::launch_signs(c->d_x[cur0], c->d_sgn[cur0], NR, st);
    for (int grp = 0; grp < ngroups && err == cudaSuccess; ++grp) {
      int cur = cur0;
      a.tile0 = ngroups > 1 ? grp : 0;
      for (int32_t k = 0; k < steps && err == cudaSuccess; ++k) {
        if (ngroups > 1) {
          a.k = k;
          a.xin = c->d_x[cur];
          a.xout = c->d_x[cur ^ 1];
          err = sbd::launch_step(variant, c->jbf16, tg, a, st);
        } else {
          err = launch(k, cur, st);
        }
        cur ^= 1;
      }
    }
    a.tile0 = 0;
    return err;
  };
  std::vector<int64_t> key;
  if (c->use_graph && steps >= 8) {
    int32_t a0b = 0, dtb = 0;
    memcpy(&a0b, &a.a0, 4);
    memcpy(&dtb, &a.dt, 4);
    key = {variant, steps, c->R, c->cur, a0b, dtb, (int64_t)(intptr_t)sched, t.G, tiled, a.rpc,
           t.tiles, a.unroll, sgn, ngroups, streamed, rw, rw_nch, ra.cta_order != nullptr,
           a.cta_order != nullptr, a.r1_lanes, fac, frw};
  }
  GraphCache& gc = c->graph;
  const bool replay = !key.empty() && gc.exec && gc.key == key;
  const bool capture = !key.empty() && !replay && gc.seen == key;
  if (!replay && !capture) {
    if (!key.empty()) gc.seen = key;
    SB_CUDA(launch_all(c->cur, stream));
    if ((steps & 1) && !x_inplace) c->cur ^= 1;
    if (c->l2_persist && win_max) {  // leave the caller's stream without our window
      cudaStreamAttrValue v = {};
      v.accessPolicyWindow.num_bytes = 0;
      SB_CUDA(cudaStreamSetAttribute(stream, cudaStreamAttributeAccessPolicyWindow, &v));
    }
    return SB_OK;
  }
  if (capture) {
    gc.reset();
    cudaGraph_t g = nullptr;
    SB_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = launch_all(c->cur, c->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    SB_CUDA(err);
    SB_CUDA(e2);
    cudaError_t e3 = cudaGraphInstantiate(&gc.exec, g, 0);
    cudaGraphDestroy(g);
    SB_CUDA(e3);
    gc.key = key;
  }
  SB_CUDA(cudaGraphLaunch(gc.exec, stream));
  if ((steps & 1) && !x_inplace) c->cur ^= 1;
  return SB_OK;
}

// Energies of R replicas (from the current x, or from d_spins) into d_Eall, arg-min into
// d_bestE / d_bestr.
sb_status readout(sb_ctx* c, const int8_t* d_spins, int32_t R, cudaStream_t s) {
  sb_status st = ensure_readout(c, R);
  if (st) return st;
  const sbd::Tiling t = sbd::make_tiling(R);
  sbd::EnergyArgs a;
  a.rowptr = c->d_rowptr;
  a.col = c->d_col;
  a.qval = c->d_qval;
  a.qlin = c->d_qlin;
  a.x = d_spins ? nullptr : c->d_x[c->cur];
  a.spins = d_spins;
  a.blk_row = c->d_blk_row;
  a.nblk = c->nblk;
  a.n = c->n;
  a.R = R;
  a.G = t.G;
  a.partial = c->d_partial;
  a.nnz = c->nnz;
  SB_CUDA(sbd::launch_energy_partial(t, a, s));
  SB_CUDA(sbd::launch_energy_reduce(c->d_partial, c->d_ev_blk0, c->E, R, c->d_Eall, s));
  SB_CUDA(sbd::launch_argmin(c->d_Eall, c->E, R, c->d_bestE, c->d_bestr, s));
  return SB_OK;
}

}  // namespace

extern "C" {

const char* sb_last_error(void) { return sbh::g_err.c_str(); }
const char* sb_version(void) { return "sbtrack-gb300 0.1 (sm_103a)"; }

sb_status sb_create(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                    const double* qval, const double* qlin, sb_jprec prec, sb_ctx** out) {
  if (!out) {
    set_error("sb_create: null output pointer");
    return SB_ERR_ARG;
  }
  int32_t ns[1] = {n};
  int64_t zs[1] = {nnz};
  return sb_create_batch(1, ns, zs, rowptr, col, qval, qlin, prec, out);
}

sb_status sb_create_batch(int32_t n_events, const int32_t* n_per_event,
                          const int64_t* nnz_per_event, const int32_t* rowptr,
                          const int32_t* col, const double* qval, const double* qlin,
                          sb_jprec prec, sb_ctx** out) {
  return sbh::guarded("sb_create_batch", [&]() -> sb_status {
    if (!out) {
      set_error("sb_create_batch: null output pointer");
      return SB_ERR_ARG;
    }
    *out = nullptr;
    if (n_events < 1 || !n_per_event || !nnz_per_event || !rowptr || !qlin ||
        (prec != SB_J_FP32 && prec != SB_J_BF16)) {
      set_error("sb_create: invalid argument (event count, null pointer or precision)");
      return SB_ERR_ARG;
    }
    int64_t ntot = 0, ztot = 0;
    for (int32_t e = 0; e < n_events; ++e) {
      if (n_per_event[e] < 1 || nnz_per_event[e] < 0) {
        set_error("sb_create: every event needs n >= 1 and nnz >= 0");
        return SB_ERR_ARG;
      }
      ntot += n_per_event[e];
      ztot += nnz_per_event[e];
    }
    if (ntot >= 0x7FFFFFFFll || ztot >= 0x7FFFFFFFll) {
      set_error("sb_create: total rows and nonzeros must stay below 2^31 - 1");
      return SB_ERR_ARG;
    }
    if (ztot > 0 && (!col || !qval)) {
      set_error("sb_create: null CSR arrays");
      return SB_ERR_ARG;
    }
    // validate each event and build the global CSR (global column indices);
    // several events: one event per task, tasks on the host threads
    std::vector<int32_t> grp((size_t)ntot + 1), gcol((size_t)ztot);
    std::vector<int32_t> ev_row0(n_events + 1);
    std::vector<int64_t> rp_off(n_events + 1, 0), z_off(n_events + 1, 0);
    for (int32_t e = 0; e < n_events; ++e) {
      ev_row0[e + 1] = ev_row0[e] + n_per_event[e];
      rp_off[e + 1] = rp_off[e] + n_per_event[e] + 1;
      z_off[e + 1] = z_off[e] + nnz_per_event[e];
    }
    std::vector<sb_status> est(n_events, SB_OK);
    std::vector<std::string> emsg(n_events);
    auto one_event = [&](int32_t e, bool threads) {
      const int32_t ne = n_per_event[e];
      const int64_t ze = nnz_per_event[e], zo = z_off[e];
      const int32_t r0 = ev_row0[e];
      const int32_t* rp = rowptr + rp_off[e];
      est[e] = validate_csr(ne, ze, rp, col + zo, qval + zo, qlin + r0, threads);
      if (est[e]) {
        emsg[e] = sbh::g_err;
        return;
      }
      for (int32_t i = 0; i < ne; ++i) grp[(size_t)r0 + i] = (int32_t)(zo + rp[i]);
      for (int64_t p = 0; p < ze; ++p) gcol[(size_t)(zo + p)] = (int32_t)(col[zo + p] + r0);
    };
    if (n_events == 1) {
      one_event(0, true);
    } else if (!parallel_parts(n_events, std::min(n_events, 256), [&](int, int64_t b, int64_t e) {
                 for (int64_t t = b; t < e; ++t) one_event((int32_t)t, false);
               }, 2)) {
      set_error("sb_create: host allocation failed");
      return SB_ERR_OOM;
    }
    for (int32_t e = 0; e < n_events; ++e)
      if (est[e]) {
        set_error(n_events > 1 ? "event " + std::to_string(e) + ": " + emsg[e] : emsg[e]);
        return est[e];
      }
    grp[ntot] = (int32_t)ztot;
    sb_ctx* c = new (std::nothrow) sb_ctx;
    if (!c) {
      set_error("sb_create: host allocation failed");
      return SB_ERR_OOM;
    }
    c->E = n_events;
    c->n = (int32_t)ntot;
    c->nnz = ztot;
    c->jbf16 = prec == SB_J_BF16;
    c->ev_row0 = ev_row0;
    c->ev_nnz.assign(nnz_per_event, nnz_per_event + n_events);
    sb_status st = create_common(c, grp.data(), gcol.data(), qval, qlin);
    c->h_rowptr.swap(grp);
    c->h_col.swap(gcol);
    if (st) {
      free_all(c);
      delete c;
      return st;
    }
    *out = c;
    return SB_OK;
  });
}

void sb_destroy(sb_ctx* ctx) {
  if (!ctx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->l2_raised) l2_persist_off(ctx);
  free_all(ctx);
  cudaSetDevice(prev);
  delete ctx;
}

int32_t sb_num_events(const sb_ctx* ctx) { return ctx ? ctx->E : 0; }
int32_t sb_total_rows(const sb_ctx* ctx) { return ctx ? ctx->n : 0; }

sb_status sb_info(const sb_ctx* ctx, int32_t e, int32_t* n, int64_t* nnz, double* offset,
                  double* sigma_j, double* c0_auto) {
  if (!ctx || e < 0 || e >= ctx->E) {
    set_error("sb_info: null context or event out of range");
    return SB_ERR_ARG;
  }
  if (n) *n = ctx->ev_row0[e + 1] - ctx->ev_row0[e];
  if (nnz) *nnz = ctx->ev_nnz[e];
  if (offset) *offset = ctx->offset[e];
  if (sigma_j) *sigma_j = ctx->sigma[e];
  if (c0_auto) *c0_auto = ctx->c0_auto[e];
  return SB_OK;
}

int32_t sb_checked_build(void) { return SB_CHECKED ? 1 : 0; }

sb_status sb_check_bounds(uint64_t* first) {
  return sbh::guarded("sb_check_bounds", [&]() -> sb_status {
    if (!first) {
      set_error("sb_check_bounds: first must not be NULL");
      return SB_ERR_ARG;
    }
    *first = 0;
    if (!SB_CHECKED) return SB_OK;
    SB_CUDA(cudaDeviceSynchronize());
    unsigned long long w[3] = {0, 0, 0};
    SB_CUDA(sbd::chk_read_kernels(&w[0]));
    SB_CUDA(sbd::chk_read_factor(&w[1]));
    SB_CUDA(sbd::chk_read_rw(&w[2]));
    static const char* const kModule[3] = {"step / energy kernels", "factored kernels",
                                            "row-group kernel"};
    static const char* const kSite[6] = {"?", "CSR column", "row-pointer pair", "U row",
                                         "group member", "row-group union column"};
    for (int m = 0; m < 3; ++m) {
      if (!w[m]) continue;
      const uint32_t site = (uint32_t)(w[m] >> 32), idx = (uint32_t)w[m];
      *first = ((uint64_t)(m + 1) << 48) | ((uint64_t)(site & 0xffff) << 32) | idx;
      set_error(std::string("sb_check_bounds: ") + kModule[m] + ": " +
                (site < 6 ? kSite[site] : "?") + " " + std::to_string((int32_t)idx) +
                " outside its array");
      return SB_ERR_BOUNDS;
    }
    return SB_OK;
  });
}

sb_status sb_step_info(const sb_ctx* ctx, int32_t* rows_per_warp, int64_t* union_entries) {
  if (!ctx) {
    set_error("sb_step_info: null context");
    return SB_ERR_ARG;
  }
  if (rows_per_warp) *rows_per_warp = ctx->rw_built;
  if (union_entries) *union_entries = ctx->rw_built ? ctx->rw_E : 0;
  return SB_OK;
}

sb_status sb_set_factor(sb_ctx* ctx, int32_t n_ids, int32_t k, const int32_t* member,
                        const uint8_t* couple, double w) {
  return sbh::guarded("sb_set_factor", [&]() -> sb_status {
    if (!ctx) {
      set_error("sb_set_factor: null context");
      return SB_ERR_ARG;
    }
    if (!member && !couple && n_ids == 0) {  // remove the factor
      free_factor(ctx);
      return SB_OK;
    }
    return set_factor(ctx, n_ids, k, member, couple, w);
  });
}

sb_status sb_factor_info(const sb_ctx* ctx, int64_t* out) {
  if (!ctx || !out) {
    set_error("sb_factor_info: null argument");
    return SB_ERR_ARG;
  }
  out[0] = ctx->fac_set ? 1 : 0;
  out[1] = ctx->fac_rows;
  out[2] = ctx->fac_rnnz;
  out[3] = ctx->fac_urows;
  out[4] = ctx->fac_ng;
  out[5] = ctx->fac_members;
  out[6] = ctx->fac_maxcount;
  return SB_OK;
}

sb_status sb_gather_probe(int64_t array_bytes, int32_t row_bytes, int32_t repeats, uint64_t seed,
                          double* out_bytes_per_s, void* stream) {
  return sbh::guarded("sb_gather_probe", [&]() -> sb_status {
    if (row_bytes <= 0 || row_bytes % 512 != 0 || array_bytes < 2LL * row_bytes || repeats < 1 ||
        !out_bytes_per_s) {
      set_error("sb_gather_probe: row_bytes a positive multiple of 512, at least two rows, "
                "repeats >= 1, out_bytes_per_s not NULL");
      return SB_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t rows = array_bytes / row_bytes;
    // about 64 reads per row, at most 2^23 reads, an even count
    const int64_t count = std::min<int64_t>(int64_t(1) << 23, std::max<int64_t>(rows * 64, 2)) & ~int64_t(1);
    std::vector<int32_t> idx((size_t)count);
    uint64_t z = seed;
    for (int64_t i = 0; i < count; ++i) {  // splitmix64
      z += 0x9E3779B97F4A7C15ull;
      uint64_t v = z;
      v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
      v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
      v ^= v >> 31;
      idx[(size_t)i] = (int32_t)(v % (uint64_t)rows);
    }
    int dev = 0, sms = 0;
    SB_CUDA(cudaGetDevice(&dev));
    SB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int per = sbd::gather_probe_blocks_per_sm();
    if (per <= 0) {
      set_error("sb_gather_probe: occupancy query failed");
      return SB_ERR_CUDA;
    }
    const int grid = sms * per;
    const size_t nwarps = (size_t)grid * sbd::gather_probe_block() / 32;
    float4* a = nullptr;
    int32_t* d_idx = nullptr;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
      dfree(a);
      dfree(d_idx);
      dfree(out);
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
    };
    sb_status st;
    if ((st = dalloc(&a, (size_t)rows * row_bytes / 16)) || (st = dalloc(&d_idx, (size_t)count)) ||
        (st = dalloc(&out, nwarps))) {
      cleanup();
      return st;
    }
    cudaError_t e = cudaMemsetAsync(a, 0, (size_t)rows * row_bytes, s);
    if (e == cudaSuccess) e = cudaMemcpy(d_idx, idx.data(), (size_t)count * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 3.0e38f;
    for (int t = 0; t <= repeats && e == cudaSuccess; ++t) {  // the first launch warms up
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess)
        e = sbd::launch_gather_probe(a, rows, row_bytes / 16, d_idx, count, out, grid, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && t > 0) best_ms = std::min(best_ms, ms);
    }
    cleanup();
    SB_CUDA(e);
    *out_bytes_per_s = (double)count * row_bytes / (best_ms * 1e-3);
    return SB_OK;
  });
}

sb_status sb_run(sb_ctx* ctx, sb_variant variant, double a0, double c0, double dt,
                 int32_t steps, int32_t replicas, uint64_t seed, const float* a_sched,
                 void* stream) {
  return sbh::guarded("sb_run", [&]() -> sb_status {
    sb_status st = check_run_args(ctx, variant, a0, c0, dt, steps);
    if (st) return st;
    if (replicas < 1 || replicas > 65535) {
      set_error("sb_run: replicas must be in [1, 65535]");
      return SB_ERR_ARG;
    }
    if ((size_t)ctx->n * (size_t)replicas >= ((size_t)1 << 40)) {
      set_error("sb_run: state too large");
      return SB_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_state(ctx, replicas))) return st;
    const float* sched = a_sched;
    if (!sched && steps > 0) {
      if (ctx->sched_len != steps || ctx->sched_a0 != a0) {
        dfree(ctx->d_sched);
        if ((st = dalloc(&ctx->d_sched, steps))) return st;
        SB_CUDA(sbd::launch_linear_schedule(ctx->d_sched, steps, a0, s));
        ctx->sched_len = steps;
        ctx->sched_a0 = a0;
      }
      sched = ctx->d_sched;
    }
    SB_CUDA(sbd::launch_set_c0(ctx->d_c0ev, ctx->d_c0auto, c0, ctx->E, s));
    ctx->cur = 0;
    SB_CUDA(sbd::launch_init(ctx->d_x[0], ctx->d_y, ctx->d_row_event, ctx->d_ev_row0, ctx->n,
                             ctx->R, seed, s));
    ctx->have_state = true;
    return enqueue_steps(ctx, variant, a0, dt, steps, sched, s);
  });
}

sb_status sb_advance(sb_ctx* ctx, sb_variant variant, double a0, double c0, double dt,
                     int32_t steps, const float* a_sched, void* stream) {
  return sbh::guarded("sb_advance", [&]() -> sb_status {
    sb_status st = check_run_args(ctx, variant, a0, c0, dt, steps);
    if (st) return st;
    if (!ctx->have_state) {
      set_error("sb_advance: no state (call sb_run or sb_set_state first)");
      return SB_ERR_STATE;
    }
    if (steps > 0 && !a_sched) {
      set_error("sb_advance: a_sched is required");
      return SB_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    SB_CUDA(sbd::launch_set_c0(ctx->d_c0ev, ctx->d_c0auto, c0, ctx->E, s));
    return enqueue_steps(ctx, variant, a0, dt, steps, a_sched, s);
  });
}

sb_status sb_set_state(sb_ctx* ctx, const float* x, const float* y, int32_t replicas,
                       int32_t on_device) {
  return sbh::guarded("sb_set_state", [&]() -> sb_status {
    if (!ctx || !x || !y || replicas < 1 || replicas > 65535) {
      set_error("sb_set_state: invalid argument");
      return SB_ERR_ARG;
    }
    sb_status st = ensure_state(ctx, replicas);
    if (st) return st;
    const size_t bytes = (size_t)ctx->n * replicas * 4;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SB_CUDA(cudaDeviceSynchronize());
    ctx->cur = 0;
    SB_CUDA(cudaMemcpy(ctx->d_x[0], x, bytes, k));
    SB_CUDA(cudaMemcpy(ctx->d_y, y, bytes, k));
    ctx->have_state = true;
    return SB_OK;
  });
}

sb_status sb_get_state(const sb_ctx* ctx, float* x, float* y, int32_t on_device) {
  if (!ctx || (!x && !y)) {
    set_error("sb_get_state: invalid argument");
    return SB_ERR_ARG;
  }
  if (!ctx->have_state) {
    set_error("sb_get_state: no state");
    return SB_ERR_STATE;
  }
  const size_t bytes = (size_t)ctx->n * ctx->R * 4;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  SB_CUDA(cudaDeviceSynchronize());
  sb_status st = check_wait_flag(ctx);
  if (st) return st;
  if (x) SB_CUDA(cudaMemcpy(x, ctx->d_x[ctx->cur], bytes, k));
  if (y) SB_CUDA(cudaMemcpy(y, ctx->d_y, bytes, k));
  return SB_OK;
}

sb_status sb_energy(sb_ctx* ctx, const int8_t* spins, int32_t replicas, double* out_E) {
  return sbh::guarded("sb_energy", [&]() -> sb_status {
    if (!ctx || !out_E || replicas < 1 || replicas > 65535) {
      set_error("sb_energy: invalid argument");
      return SB_ERR_ARG;
    }
    sb_status st;
    if (spins) {
      if (ctx->spins_cap_R < replicas) {
        dfree(ctx->d_spins);
        if ((st = dalloc(&ctx->d_spins, (size_t)ctx->n * replicas))) return st;
        ctx->spins_cap_R = replicas;
      }
      SB_CUDA(cudaMemcpy(ctx->d_spins, spins, (size_t)ctx->n * replicas, cudaMemcpyHostToDevice));
    } else {
      if (!ctx->have_state || ctx->R != replicas) {
        set_error("sb_energy: no current state with that replica count");
        return SB_ERR_STATE;
      }
    }
    if ((st = readout(ctx, spins ? ctx->d_spins : nullptr, replicas, 0))) return st;
    SB_CUDA(cudaDeviceSynchronize());
    if (!spins && (st = check_wait_flag(ctx))) return st;
    SB_CUDA(cudaMemcpy(out_E, ctx->d_Eall, (size_t)ctx->E * replicas * 8, cudaMemcpyDeviceToHost));
    return SB_OK;
  });
}

sb_status sb_readout_device(sb_ctx* ctx, double* d_E_all, double* d_best_E, int32_t* d_best_r,
                            uint8_t* d_T, void* stream) {
  return sbh::guarded("sb_readout_device", [&]() -> sb_status {
    if (!ctx) {
      set_error("sb_readout_device: null context");
      return SB_ERR_ARG;
    }
    if (!ctx->have_state) {
      set_error("sb_readout_device: no state");
      return SB_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    sb_status st = readout(ctx, nullptr, ctx->R, s);
    if (st) return st;
    if (d_T)
      SB_CUDA(sbd::launch_best_T(ctx->d_x[ctx->cur], ctx->d_row_event, ctx->d_bestr, ctx->n,
                                 ctx->R, d_T, s));
    if (d_E_all)
      SB_CUDA(cudaMemcpyAsync(d_E_all, ctx->d_Eall, (size_t)ctx->E * ctx->R * 8,
                              cudaMemcpyDeviceToDevice, s));
    if (d_best_E)
      SB_CUDA(cudaMemcpyAsync(d_best_E, ctx->d_bestE, ctx->E * 8, cudaMemcpyDeviceToDevice, s));
    if (d_best_r)
      SB_CUDA(cudaMemcpyAsync(d_best_r, ctx->d_bestr, ctx->E * 4, cudaMemcpyDeviceToDevice, s));
    return SB_OK;
  });
}

sb_status sb_best(sb_ctx* ctx, uint8_t* out_T, double* out_E, int32_t* out_replica) {
  return sbh::guarded("sb_best", [&]() -> sb_status {
    if (!ctx) {
      set_error("sb_best: null context");
      return SB_ERR_ARG;
    }
    sb_status st = sb_readout_device(ctx, nullptr, nullptr, nullptr, out_T ? ctx->d_T : nullptr, 0);
    if (st) return st;
    SB_CUDA(cudaDeviceSynchronize());
    if ((st = check_wait_flag(ctx))) return st;
    if (out_T) SB_CUDA(cudaMemcpy(out_T, ctx->d_T, ctx->n, cudaMemcpyDeviceToHost));
    if (out_E) SB_CUDA(cudaMemcpy(out_E, ctx->d_bestE, ctx->E * 8, cudaMemcpyDeviceToHost));
    if (out_replica)
      SB_CUDA(cudaMemcpy(out_replica, ctx->d_bestr, ctx->E * 4, cudaMemcpyDeviceToHost));
    return SB_OK;
  });
}

sb_status sb_set_weights(sb_ctx* ctx, const int8_t* cls, const double* quality, double w_q,
                         double w_c) {
  return sbh::guarded("sb_set_weights", [&]() -> sb_status {
    if (!ctx || !quality || (!cls && ctx->nnz > 0) || !std::isfinite(w_q) || !std::isfinite(w_c)) {
      set_error("sb_set_weights: invalid argument");
      return SB_ERR_ARG;
    }
    if (ctx->E != 1) {
      set_error("sb_set_weights: single-event contexts only");
      return SB_ERR_ARG;
    }
    const int32_t n = ctx->n;
    const int32_t* rp = ctx->h_rowptr.data();
    const int32_t* col = ctx->h_col.data();
    std::vector<double> qv((size_t)ctx->nnz), ql(n), nconf(n, 0.0);
    for (int32_t i = 0; i < n; ++i) {
      if (!std::isfinite(quality[i])) {
        set_error("sb_set_weights: quality not finite");
        return SB_ERR_ARG;
      }
      ql[i] = w_q * quality[i];
      for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        if (cls[p] != 0 && cls[p] != 1) {
          set_error("sb_set_weights: class tags must be 0 (consistent) or 1 (conflict)");
          return SB_ERR_ARG;
        }
        const int32_t j = col[p];
        const int32_t* f = std::lower_bound(col + rp[j], col + rp[j + 1], i);
        if (cls[rp[j] + (f - (col + rp[j]))] != cls[p]) {
          set_error("sb_set_weights: class tags are not symmetric");
          return SB_ERR_CSR;
        }
        qv[p] = cls[p] ? w_c : -1.0;
        nconf[i] += cls[p] ? 1.0 : 0.0;
      }
    }
    sb_status st;
    if (!ctx->d_cls) {
      if ((st = dalloc(&ctx->d_cls, (size_t)ctx->nnz)) || (st = dalloc(&ctx->d_quality, (size_t)n)) ||
          (st = dalloc(&ctx->d_nconf, (size_t)n)))
        return st;
    }
    SB_CUDA(cudaDeviceSynchronize());
    if (ctx->nnz) {
      SB_CUDA(cudaMemcpy(ctx->d_cls, cls, (size_t)ctx->nnz, cudaMemcpyHostToDevice));
      SB_CUDA(cudaMemcpy(ctx->d_qval, qv.data(), (size_t)ctx->nnz * 8, cudaMemcpyHostToDevice));
    }
    SB_CUDA(cudaMemcpy(ctx->d_quality, quality, (size_t)n * 8, cudaMemcpyHostToDevice));
    SB_CUDA(cudaMemcpy(ctx->d_nconf, nconf.data(), (size_t)n * 8, cudaMemcpyHostToDevice));
    SB_CUDA(cudaMemcpy(ctx->d_qlin, ql.data(), (size_t)n * 8, cudaMemcpyHostToDevice));
    double *row_off = nullptr, *row_sq = nullptr;
    if ((st = dalloc(&row_off, (size_t)n)) || (st = dalloc(&row_sq, (size_t)n))) {
      dfree(row_off);
      dfree(row_sq);
      return st;
    }
    cudaError_t e1 = sbd::launch_convert(ctx->d_rowptr, ctx->d_col, ctx->d_qval, ctx->d_qlin, n,
                                         ctx->d_J, ctx->jbf16, ctx->d_h64, ctx->d_h32, row_off,
                                         row_sq, 0);
    cudaError_t e2 = sbd::launch_event_stats(row_off, row_sq, ctx->d_ev_row0, 1, ctx->d_offset,
                                             ctx->d_sigma, ctx->d_c0auto, 0);
    cudaError_t e3 = cudaDeviceSynchronize();
    dfree(row_off);
    dfree(row_sq);
    SB_CUDA(e1);
    SB_CUDA(e2);
    SB_CUDA(e3);
    SB_CUDA(cudaMemcpy(ctx->offset.data(), ctx->d_offset, 8, cudaMemcpyDeviceToHost));
    SB_CUDA(cudaMemcpy(ctx->sigma.data(), ctx->d_sigma, 8, cudaMemcpyDeviceToHost));
    SB_CUDA(cudaMemcpy(ctx->c0_auto.data(), ctx->d_c0auto, 8, cudaMemcpyDeviceToHost));
    note_j_range(ctx);
    // the tiled kernel's packed words carry J: rebuild them
    dfree(ctx->d_blk_row0);
    dfree(ctx->d_blk_u0);
    dfree(ctx->d_ucol);
    dfree(ctx->d_own);
    if (ctx->d_tz) cudaFree(ctx->d_tz);
    ctx->d_tz = nullptr;
    ctx->graph.reset();
    if (ctx->tiles_built && (st = setup_tiles(ctx, rp, col))) return st;
    // the row-group kernel's entries carry J too
    if ((st = refill_rw(ctx))) return st;
    // the factored form's weight and residual were formed for the old couplings
    free_factor(ctx);
    ctx->have_classes = true;
    return SB_OK;
  });
}

sb_status sb_backward(sb_ctx* ctx, double a0, double c0, double dt, int32_t steps,
                      int32_t replicas, uint64_t seed, const float* a_sched, int32_t ckpt_every,
                      double* out_loss, double* out_grads, double* d_grad_sched, void* stream) {
  return sbh::guarded("sb_backward", [&]() -> sb_status {
    sb_status st = check_run_args(ctx, SB_BSB, a0, c0, dt, steps);
    if (st) return st;
    if (ctx->E != 1 || !(c0 > 0.0) || steps < 1 || ckpt_every < 1 || replicas < 1 ||
        replicas > 65535) {
      set_error("sb_backward: single event, c0 > 0, steps >= 1, ckpt_every >= 1, 1 <= R <= 65535");
      return SB_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_state(ctx, replicas))) return st;
    const int32_t n = ctx->n, R = replicas, S = steps, K = std::min(ckpt_every, steps);
    const size_t NR = (size_t)n * R;
    const int32_t n_ck = (S + K - 1) / K;
    if (!ctx->d_cls) {  // no class tags: weight-scale gradients are reported as NaN
      if ((st = dalloc(&ctx->d_cls, (size_t)ctx->nnz)) || (st = dalloc(&ctx->d_quality, (size_t)n)) ||
          (st = dalloc(&ctx->d_nconf, (size_t)n)))
        return st;
      SB_CUDA(cudaMemset(ctx->d_cls, 0, std::max<size_t>((size_t)ctx->nnz, 1)));
      SB_CUDA(cudaMemset(ctx->d_quality, 0, (size_t)n * 8));
      SB_CUDA(cudaMemset(ctx->d_nconf, 0, (size_t)n * 8));
    }
    const float* sched = a_sched;
    if (!sched) {
      if (ctx->sched_len != S || ctx->sched_a0 != a0) {
        dfree(ctx->d_sched);
        if ((st = dalloc(&ctx->d_sched, S))) return st;
        SB_CUDA(sbd::launch_linear_schedule(ctx->d_sched, S, a0, s));
        ctx->sched_len = S;
        ctx->sched_a0 = a0;
      }
      sched = ctx->d_sched;
    }
    // work memory: checkpoints for all segments but the last (recorded on the
    // way forward), one segment's recording, the adjoint state (two buffers
    // for the adjoint of y~: a reverse step reads one, writes the other)
    sb_ctx::AdjWork& w = ctx->adj;
    if (w.n != n || w.R != R || w.S != S || w.K != K) {
      free_adj(ctx);
      if ((st = dalloc(&w.ck_x, NR * (n_ck - 1))) || (st = dalloc(&w.ck_y, NR * (n_ck - 1))) ||
          (st = dalloc(&w.seg_x, NR * (K + 1))) || (st = dalloc(&w.seg_yt, NR * K)) ||
          (st = dalloc(&w.seg_f, NR * K)) || (st = dalloc(&w.seg_m, NR * K)) ||
          (st = dalloc(&w.lx, NR)) || (st = dalloc(&w.ly, NR)) || (st = dalloc(&w.lyt[0], NR)) ||
          (st = dalloc(&w.lyt[1], NR)) || (st = dalloc(&w.gh, (size_t)n)) ||
          (st = dalloc(&w.acc, 6)) || (st = dalloc(&w.ga, (size_t)S))) {
        free_adj(ctx);
        return st;
      }
      w.n = n;
      w.R = R;
      w.S = S;
      w.K = K;
    }
    float *ck_x = w.ck_x, *ck_y = w.ck_y, *seg_x = w.seg_x, *seg_yt = w.seg_yt, *seg_f = w.seg_f;
    float *lx = w.lx, *ly = w.ly;
    uint8_t* seg_m = w.seg_m;
    double *gh = w.gh, *acc = w.acc, *ga = w.ga;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
      return e == cudaSuccess;
    };
    const sbd::Tiling t = sbd::make_tiling(R);
    sbd::StepArgs a;
    a.rowptr = ctx->d_rowptr;
    a.col = ctx->d_col;
    a.J = ctx->d_J;
    a.h = ctx->d_h32;
    a.row_event = nullptr;
    a.c0_ev = ctx->d_c0ev;
    a.sched = sched;
    a.a0 = (float)a0;
    a.dt = (float)dt;
    a.dta0 = (float)(dt * a0);
    a.n = n;
    a.R = R;
    a.G = t.G;
    a.rpc = 256 / t.G;
    a.unroll = 4;
    a.tile0 = 0;
    a.nnz = ctx->nnz;
    a.ytil = nullptr;
    a.mask = nullptr;
    a.frec = nullptr;
    a.sgn_in = nullptr;
    a.sgn_out = nullptr;
    a.r1_lanes = r1_lanes_for(ctx);
    ok(sbd::launch_set_c0(ctx->d_c0ev, ctx->d_c0auto, c0, 1, s));
    ok(sbd::launch_init(ctx->d_x[0], ctx->d_y, nullptr, ctx->d_ev_row0, n, R, seed, s));
    int cur = 0;
    // forward, keeping (x, y) at the start of every segment but the last
    for (int32_t c = 0; c + 1 < n_ck && e == cudaSuccess; ++c) {
      ok(cudaMemcpyAsync(ck_x + NR * c, ctx->d_x[cur], NR * 4, cudaMemcpyDeviceToDevice, s));
      ok(cudaMemcpyAsync(ck_y + NR * c, ctx->d_y, NR * 4, cudaMemcpyDeviceToDevice, s));
      for (int32_t j = 0; j < K && e == cudaSuccess; ++j) {
        a.k = c * K + j;
        a.xin = ctx->d_x[cur];
        a.xout = ctx->d_x[cur ^ 1];
        a.y = ctx->d_y;
        ok(sbd::launch_step(SB_BSB, ctx->jbf16, t, a, s));
        cur ^= 1;
      }
    }
    // the last segment, recorded as it runs: x_k, pre-wall momentum, wall mask, J x_k
    const int32_t c_last = n_ck - 1;
    const int32_t L_last = S - c_last * K;
    auto record_segment = [&](int32_t c, int32_t L) {
      for (int32_t j = 0; j < L && e == cudaSuccess; ++j) {
        a.k = c * K + j;
        a.xin = seg_x + NR * j;
        a.xout = seg_x + NR * (j + 1);
        a.y = ctx->d_y;
        a.ytil = seg_yt + NR * j;
        a.mask = seg_m + NR * j;
        a.frec = seg_f + NR * j;
        ok(sbd::launch_step(SB_BSB, ctx->jbf16, t, a, s));
      }
      a.ytil = nullptr;
      a.mask = nullptr;
      a.frec = nullptr;
    };
    ok(cudaMemcpyAsync(seg_x, ctx->d_x[cur], NR * 4, cudaMemcpyDeviceToDevice, s));
    record_segment(c_last, L_last);
    ok(cudaMemsetAsync(gh, 0, (size_t)n * 8, s));
    ok(cudaMemsetAsync(acc, 0, 6 * 8, s));
    ok(cudaMemsetAsync(ga, 0, (size_t)S * 8, s));
    sbd::AdjArgs g;
    g.rowptr = ctx->d_rowptr;
    g.col = ctx->d_col;
    g.J = ctx->d_J;
    g.cls = ctx->d_cls;
    g.h = ctx->d_h32;
    g.quality = ctx->d_quality;
    g.nconf = ctx->d_nconf;
    g.n = n;
    g.R = R;
    g.G = t.G;
    g.a0 = (float)a0;
    g.c0 = (float)c0;
    g.dt = (float)dt;
    g.sched = sched;
    g.k = 0;
    g.x = seg_x + NR * L_last;  // x_S
    g.ytil = nullptr;
    g.mask = nullptr;
    g.frec = nullptr;
    g.lx = lx;
    g.ly = ly;
    g.lyt = w.lyt[0];
    g.gh = gh;
    g.acc = acc;
    g.ga = nullptr;
    ok(sbd::launch_adj_init(ctx->jbf16, t, g, s));
    // reverse sweep, one segment at a time: recompute it with recording (the
    // last one is recorded already), then reverse it
    for (int32_t c = n_ck - 1; c >= 0 && e == cudaSuccess; --c) {
      const int32_t L = std::min(K, S - c * K);
      if (c < c_last) {
        ok(cudaMemcpyAsync(seg_x, ck_x + NR * c, NR * 4, cudaMemcpyDeviceToDevice, s));
        ok(cudaMemcpyAsync(ctx->d_y, ck_y + NR * c, NR * 4, cudaMemcpyDeviceToDevice, s));
        record_segment(c, L);
      }
      // phase 1 (through the wall) of a segment's last step runs alone; every
      // other step's phase 1 is fused into the reverse step after it
      int lb = 0;  // lyt buffer holding the adjoint of y~ of the step being reversed
      for (int32_t j = L - 1; j >= 0 && e == cudaSuccess; --j) {
        g.k = c * K + j;
        g.x = seg_x + NR * j;
        g.ytil = seg_yt + NR * j;
        g.mask = seg_m + NR * j;
        g.frec = seg_f + NR * j;
        g.ga = ga + g.k;
        g.lyt = w.lyt[lb];
        if (j == L - 1) ok(sbd::launch_adj_phase1(g, s));
        g.mask_prev = j > 0 ? seg_m + NR * (j - 1) : nullptr;
        g.lyt_out = j > 0 ? w.lyt[lb ^ 1] : nullptr;
        ok(sbd::launch_adj_phase2(ctx->jbf16, t, g, s));
        g.mask_prev = nullptr;
        g.lyt_out = nullptr;
        lb ^= 1;
      }
    }
    ok(sbd::launch_adj_final(g, acc + 4, s));
    if (d_grad_sched) ok(cudaMemcpyAsync(d_grad_sched, ga, (size_t)S * 8, cudaMemcpyDeviceToDevice, s));
    ok(cudaStreamSynchronize(s));
    double h_acc[6] = {0, 0, 0, 0, 0, 0};
    ok(cudaMemcpy(h_acc, acc, sizeof(h_acc), cudaMemcpyDeviceToHost));
    ctx->have_state = false;  // x holds x_S but y was reused by the recomputation
    SB_CUDA(e);
    if (out_loss) *out_loss = h_acc[0];
    if (out_grads) {
      const double nan = std::nan("");
      out_grads[0] = h_acc[1];
      out_grads[1] = h_acc[2];
      out_grads[2] = ctx->have_classes ? h_acc[4] : nan;
      out_grads[3] = ctx->have_classes ? h_acc[3] + h_acc[5] : nan;
    }
    return SB_OK;
  });
}

sb_status sb_set_option(sb_ctx* ctx, int32_t key, int64_t value);

sb_status sb_autotune(sb_ctx* ctx, sb_variant variant, int32_t replicas, int32_t trial_steps,
                      int32_t* out_cfg, float* out_us_per_step, void* stream) {
  return sbh::guarded("sb_autotune", [&]() -> sb_status {
    if (!ctx || replicas < 1 || replicas > 65535 || trial_steps < 1 || trial_steps > 100000) {
      set_error("sb_autotune: invalid argument");
      return SB_ERR_ARG;
    }
    sb_status st = check_run_args(ctx, variant, 1.0, 0.0, 0.5, trial_steps);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // candidates: (tiled, replica-tile width, rows per CTA); invalid ones are skipped
    struct Cand {
      int tiled, rt, rpc, unroll, groups, l2, rw, fac;
    };
    std::vector<Cand> cands = {
        {0, 0, 0, 4, 1, 0, 0, 0},  {0, 0, 32, 4, 1, 0, 0, 0},  {0, 0, 0, 4, 1, 1, 0, 0},
        {0, 0, 32, 4, 1, 1, 0, 0}, {0, 128, 0, 4, 1, 0, 0, 0}, {0, 128, 32, 4, 1, 0, 0, 0},
        {0, 64, 0, 4, 1, 0, 0, 0}, {0, 32, 0, 4, 1, 0, 0, 0},  {0, 0, 0, 4, 2, 0, 0, 0},
        {0, 0, 32, 4, 2, 0, 0, 0}, {0, 0, 0, 4, 4, 0, 0, 0},   {1, 0, 0, 4, 1, 0, 0, 0},
        {0, 0, 0, 4, 1, 0, 2, 0},  {0, 0, 32, 4, 1, 0, 2, 0},  {0, 0, 64, 4, 1, 0, 2, 0},
        {0, 128, 0, 4, 1, 0, 2, 0}, {0, 0, 0, 4, 1, 0, 4, 0},  {0, 0, 64, 4, 1, 0, 4, 0},
        {0, 128, 0, 4, 1, 0, 4, 0}};
    // the factored product (when set and not switched off) is one more candidate
    const int fac_allowed = ctx->fac_set && ctx->fac_use != 0;
    // (aSB / bSB: through the row-group kernel when rows per warp are left
    // automatic, or the dedicated factored kernel with rows per warp off)
    if (fac_allowed) {
      cands.insert(cands.begin(), Cand{0, 0, 0, 4, 1, 0, 0, 1});
      cands.insert(cands.begin(), Cand{0, 0, 0, 4, 1, 0, -1, 1});
    }
    const int keep_graph = ctx->use_graph;
    ctx->use_graph = 0;
    if ((st = ensure_state(ctx, replicas))) return st;
    float* sched = nullptr;
    if ((st = dalloc(&sched, (size_t)trial_steps))) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best_us = 3.0e38f;
    int best = 0;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = sbd::launch_linear_schedule(sched, trial_steps, 1.0, s);
    for (size_t k = 0; k < cands.size() && err == cudaSuccess; ++k) {
      const Cand& c = cands[k];
      if (c.tiled) {
        if (replicas % sbd::kTileRT != 0) continue;
        if ((st = ensure_tiles(ctx))) break;
        if (!ctx->tiled_ok) continue;
      }
      if (c.rt && (replicas % c.rt != 0)) continue;
      if (c.rw > 0 && replicas % 128 != 0) continue;
      if (c.groups > 1) {
        const int rt = replicas / c.groups;
        if (replicas % (4 * c.groups) != 0 || rt > 128 || ((rt / 4) & (rt / 4 - 1)) != 0) continue;
      }
      ctx->use_tiled = c.tiled;
      ctx->step_rt = c.rt;
      ctx->step_rpc = c.rpc;
      ctx->step_unroll = c.unroll;
      ctx->groups = c.groups;
      ctx->rw_rows = c.rw;
      ctx->fac_use = c.fac ? -1 : 0;
      if ((st = c.l2 ? l2_persist_on(ctx) : l2_persist_off(ctx))) break;
      ctx->l2_persist = c.l2;
      ctx->graph.reset();
      if ((st = sb_run(ctx, variant, 1.0, 0.0, 0.5, 0, replicas, 12345, nullptr, stream))) break;
      if ((st = enqueue_steps(ctx, variant, 1.0, 0.5, std::min(trial_steps, 4), sched, s))) break;
      err = cudaEventRecord(e0, s);
      if (err != cudaSuccess) break;
      if ((st = enqueue_steps(ctx, variant, 1.0, 0.5, trial_steps, sched, s))) break;
      err = cudaEventRecord(e1, s);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      const float us = ms * 1000.f / trial_steps;
      if (err == cudaSuccess && us < best_us) {
        best_us = us;
        best = (int)k;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(sched);
    ctx->use_graph = keep_graph;
    ctx->have_state = false;
    if (st) return st;
    SB_CUDA(err);
    ctx->use_tiled = cands[best].tiled;
    ctx->step_rt = cands[best].rt;
    ctx->step_rpc = cands[best].rpc;
    ctx->step_unroll = cands[best].unroll;
    ctx->groups = cands[best].groups;
    ctx->l2_persist = cands[best].l2;
    if ((st = ctx->l2_persist ? l2_persist_on(ctx) : l2_persist_off(ctx))) return st;
    ctx->rw_rows = cands[best].rw;
    ctx->fac_use = cands[best].fac ? -1 : (fac_allowed ? 0 : ctx->fac_use);
    ctx->graph.reset();
    if (out_cfg) {
      out_cfg[0] = cands[best].tiled;
      out_cfg[1] = cands[best].rt;
      out_cfg[2] = cands[best].rpc;
      out_cfg[3] = cands[best].unroll;
      out_cfg[4] = cands[best].groups;
      out_cfg[5] = cands[best].l2;
      out_cfg[6] = cands[best].rw;
      out_cfg[7] = cands[best].fac;
    }
    if (out_us_per_step) *out_us_per_step = best_us;
    return SB_OK;
  });
}

sb_status sb_set_option(sb_ctx* ctx, int32_t key, int64_t value) {
  return sbh::guarded("sb_set_option", [&]() -> sb_status {
    if (!ctx) {
      set_error("sb_set_option: null context");
      return SB_ERR_ARG;
    }
    switch (key) {
      case 0:  // SB_OPT_GRAPH
        ctx->use_graph = value != 0;
        if (!ctx->use_graph) ctx->graph.reset();
        return SB_OK;
      case 1:  // SB_OPT_TILED
        ctx->use_tiled = value != 0;
        ctx->graph.reset();
        return SB_OK;
      case 2:  // SB_OPT_STEP_RT
        if (value != 0 && (value % 4 != 0 || value > 128 || value < 4 ||
                           ((value / 4) & (value / 4 - 1)) != 0)) {
          set_error("sb_set_option: SB_OPT_STEP_RT must be 0 or 4 * (a power of two <= 32)");
          return SB_ERR_ARG;
        }
        ctx->step_rt = (int)value;
        ctx->graph.reset();
        return SB_OK;
      case 3:  // SB_OPT_STEP_RPC
        if (value < -1 || value > (1 << 20)) {
          set_error("sb_set_option: SB_OPT_STEP_RPC out of range");
          return SB_ERR_ARG;
        }
        ctx->step_rpc = (int)value;
        ctx->graph.reset();
        return SB_OK;
      case 4:  // SB_OPT_STEP_UNROLL
        if (value != 4) {
          set_error("sb_set_option: SB_OPT_STEP_UNROLL must be 4 (8 measured slower and was removed)");
          return SB_ERR_ARG;
        }
        ctx->step_unroll = (int)value;
        ctx->graph.reset();
        return SB_OK;
      case 5:  // SB_OPT_DSB_SIGNS
        ctx->dsb_signs = value != 0;
        ctx->graph.reset();
        return SB_OK;
      case 7: {  // SB_OPT_L2_PERSIST
        const sb_status st = value ? l2_persist_on(ctx) : l2_persist_off(ctx);
        if (st) return st;
        ctx->l2_persist = value != 0;
        ctx->graph.reset();
        return SB_OK;
      }
      case 9:  // SB_OPT_ROWS_PER_WARP
        if (value != -1 && value != 0 && value != 2 && value != 4) {
          set_error("sb_set_option: SB_OPT_ROWS_PER_WARP must be -1, 0, 2 or 4");
          return SB_ERR_ARG;
        }
        ctx->rw_rows = (int)value;
        ctx->graph.reset();
        return SB_OK;
      case 11:  // SB_OPT_R1_LANES
        if (value != -1 && value != 0 && value != 8 && value != 16 && value != 32) {
          set_error("sb_set_option: SB_OPT_R1_LANES must be -1, 0, 8, 16 or 32");
          return SB_ERR_ARG;
        }
        ctx->r1_lanes = (int)value;
        ctx->graph.reset();
        return SB_OK;
      case 10:  // SB_OPT_HEAVY_FIRST
        if (value < -1 || value > 1) {
          set_error("sb_set_option: SB_OPT_HEAVY_FIRST must be -1, 0 or 1");
          return SB_ERR_ARG;
        }
        ctx->rw_heavy_first = (int)value;
        ctx->graph.reset();
        return SB_OK;
      case 8:  // SB_OPT_STREAM
        ctx->use_stream = value != 0;
        ctx->graph.reset();
        return SB_OK;
      case 15:  // SB_OPT_TEST_BAD_COL (bounds-checked build only)
        if (!SB_CHECKED) {
          set_error("sb_set_option: SB_OPT_TEST_BAD_COL needs the bounds-checked build");
          return SB_ERR_ARG;
        }
        if (value < 0 || value >= ctx->nnz) {
          set_error("sb_set_option: SB_OPT_TEST_BAD_COL must be a CSR entry in [0, nnz)");
          return SB_ERR_ARG;
        }
        {
          const int32_t bad = ctx->n + 7;
          SB_CUDA(cudaMemcpy(ctx->d_col + value, &bad, sizeof(bad), cudaMemcpyHostToDevice));
        }
        ctx->graph.reset();
        return SB_OK;
      case 14:  // SB_OPT_FACTOR
        if (value < -1 || value > 1) {
          set_error("sb_set_option: SB_OPT_FACTOR must be -1, 0 or 1");
          return SB_ERR_ARG;
        }
        ctx->fac_use = (int)value;
        ctx->graph.reset();
        return SB_OK;
      case 12:  // SB_OPT_WAIT_NS
        if (value < 1000 || value > 60000000000ll) {
          set_error("sb_set_option: SB_OPT_WAIT_NS must be in [1e3, 6e10] nanoseconds");
          return SB_ERR_ARG;
        }
        ctx->wait_ns = (unsigned long long)value;
        ctx->graph.reset();
        return SB_OK;
      case 13:  // SB_OPT_TEST_SKIP_STAGE
        if (value < -1 || value > (1 << 30)) {
          set_error("sb_set_option: SB_OPT_TEST_SKIP_STAGE must be -1 or a stage index");
          return SB_ERR_ARG;
        }
        ctx->skip_stage = (int32_t)value;
        ctx->graph.reset();
        return SB_OK;
      case 6:  // SB_OPT_REPLICA_GROUPS
        if (value < 1 || value > 64) {
          set_error("sb_set_option: SB_OPT_REPLICA_GROUPS must be in [1, 64]");
          return SB_ERR_ARG;
        }
        ctx->groups = (int)value;
        ctx->graph.reset();
        return SB_OK;
      default:
        set_error("sb_set_option: unknown key");
        return SB_ERR_ARG;
    }
  });
}

}  // extern "C"
