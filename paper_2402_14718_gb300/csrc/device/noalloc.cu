// sb_energy_noalloc: the FP64 QUBO energy readout (energies of R replicas,
// arg-min, best energy) for callers that must not allocate device memory.
//
// Its scratch -- the block row table and the per-block partial energies that
// the readout kernels need between their two passes -- lives in the
// file-scope array g_scratch below (kScratchBytes per GPU). This file is its
// own module (the library is linked without relocatable device code), and
// CUDA loads modules lazily: the first call on a device loads the module and
// commits the array there (a driver allocation that can synchronise); from
// then on the array stays committed in that context until the process exits
// or the context is destroyed. Nothing here calls cudaMalloc, cudaFree or any
// allocating library routine.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../../include/sb.h"
#include "kernels.cuh"

namespace sbh {
void set_error(const std::string& msg);
}

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up with the device current (in host
// code the symbol is only a host-side stand-in). The address belongs to the
// context the module was loaded in: it is cached per device together with
// that context, and looked up again when the current context differs (after
// cudaDeviceReset the primary context, and with it the module, is new).
struct ScratchSlot {
  CUcontext ctx;
  void* addr;
};
ScratchSlot g_slot[kMaxDevices];
std::mutex g_scratch_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry point (no link against
// libcuda, so the library still loads on machines without a driver). Writes
// NULL when no context is current yet.
sb_status current_context(CUcontext* out) {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      sbh::set_error(std::string("sb_energy_noalloc: cuCtxGetCurrent entry point: ") +
                     cudaGetErrorString(e));
      return SB_ERR_CUDA;
    }
    fn = reinterpret_cast<CtxGetCurrentFn>(p);
  }
  CUcontext c = nullptr;
  if (fn(&c) != CUDA_SUCCESS) {
    sbh::set_error("sb_energy_noalloc: cuCtxGetCurrent failed");
    return SB_ERR_CUDA;
  }
  *out = c;
  return SB_OK;
}

sb_status symbol_address(void** p) {
  cudaError_t e = cudaGetSymbolAddress(p, g_scratch);
  if (e != cudaSuccess || !*p) {
    sbh::set_error(std::string("sb_energy_noalloc: cudaGetSymbolAddress: ") +
                   cudaGetErrorString(e));
    return SB_ERR_CUDA;
  }
  return SB_OK;
}

// The scratch address in the calling thread's current context (the caller's
// own context if one is current, else the device's primary context, which
// the runtime creates on first use).
sb_status scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    sbh::set_error(std::string("sb_energy_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return SB_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    sbh::set_error("sb_energy_noalloc: device ordinal out of range");
    return SB_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  CUcontext ctx = nullptr;
  sb_status st = current_context(&ctx);
  if (st) return st;
  void* p = nullptr;
  if (!ctx) {  // nothing current yet: the runtime's first call makes the primary context
    st = symbol_address(&p);
    if (st) return st;
    st = current_context(&ctx);
    if (st) return st;
    if (!ctx) {
      sbh::set_error("sb_energy_noalloc: no current CUDA context");
      return SB_ERR_CUDA;
    }
    g_slot[dev].addr = p;
    g_slot[dev].ctx = ctx;
  } else if (!g_slot[dev].addr || g_slot[dev].ctx != ctx) {
    st = symbol_address(&p);
    if (st) return st;
    g_slot[dev].addr = p;
    g_slot[dev].ctx = ctx;
  }
  *out = g_slot[dev].addr;
  return SB_OK;
}

// Uniform row blocks of `rows` rows: blk_row[b] = min(b * rows, n), one event.
__global__ void k_fill_block_table(int32_t* blk_row, int32_t* ev_blk0, int32_t n, int32_t rows,
                                   int32_t nblk) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= nblk; b += gridDim.x * blockDim.x) {
    const long long r = (long long)b * rows;
    blk_row[b] = (int32_t)(r < n ? r : n);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ev_blk0[0] = 0;
    ev_blk0[1] = nblk;
  }
}

}  // namespace

extern "C" sb_status sb_energy_noalloc(int32_t n, const int32_t* d_rowptr, const int32_t* d_col,
                                       const double* d_qval, const double* d_qlin,
                                       const float* d_x, const int8_t* d_spins, int32_t replicas,
                                       double* d_E, double* d_best_E, int32_t* d_best_r,
                                       void* stream) {
  if (n < 1 || !d_rowptr || !d_col || !d_qval || !d_qlin || !d_E || replicas < 1 ||
      replicas > 65535 ||
      ((d_x == nullptr) == (d_spins == nullptr)) || ((d_best_E == nullptr) != (d_best_r == nullptr))) {
    sbh::set_error(
        "sb_energy_noalloc: need n >= 1, rowptr, col, qval, qlin, E, 1 <= replicas <= 65535, "
        "exactly one of "
        "x / spins, and best_E and best_r both given or both NULL");
    return SB_ERR_ARG;
  }
  const sbd::Tiling t = sbd::make_tiling(replicas);
  const int32_t rows = 256 / t.G > 64 ? 256 / t.G : 64;
  const long long nblk = ((long long)n + rows - 1) / rows;
  // scratch layout: [blk_row: nblk + 1 int32][ev_blk0: 2 int32] ... [partial: nblk x R double]
  const size_t table_bytes = (size_t)(nblk + 1 + 2) * sizeof(int32_t);
  const size_t partial_off = (table_bytes + 255) & ~size_t(255);
  const size_t need = partial_off + (size_t)nblk * (size_t)replicas * sizeof(double);
  if (need > kScratchBytes) {
    sbh::set_error("sb_energy_noalloc: " + std::to_string(n) + " rows x " +
                   std::to_string(replicas) + " replicas need " + std::to_string(need) +
                   " bytes of scratch; the static scratch holds " +
                   std::to_string(kScratchBytes) + " bytes (use sb_energy / sb_readout_device)");
    return SB_ERR_ARG;
  }
  void* base = nullptr;
  sb_status st = scratch_address(&base);
  if (st) return st;
  unsigned char* s = static_cast<unsigned char*>(base);
  int32_t* blk_row = reinterpret_cast<int32_t*>(s);
  int32_t* ev_blk0 = blk_row + nblk + 1;
  double* partial = reinterpret_cast<double*>(s + partial_off);
  cudaStream_t cs = (cudaStream_t)stream;

  const int grid = (int)((nblk + 1 + 255) / 256);
  k_fill_block_table<<<grid, 256, 0, cs>>>(blk_row, ev_blk0, n, rows, (int32_t)nblk);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    sbd::EnergyArgs a;
    a.rowptr = d_rowptr;
    a.col = d_col;
    a.qval = d_qval;
    a.qlin = d_qlin;
    a.x = d_x;
    a.spins = d_spins;
    a.blk_row = blk_row;
    a.nblk = (int32_t)nblk;
    a.n = n;
    a.R = replicas;
    a.G = t.G;
    a.partial = partial;  // every (block, replica) entry is written before it is read
    e = sbd::launch_energy_partial(t, a, cs);
  }
  if (e == cudaSuccess) e = sbd::launch_energy_reduce(partial, ev_blk0, 1, replicas, d_E, cs);
  if (e == cudaSuccess && d_best_E) e = sbd::launch_argmin(d_E, 1, replicas, d_best_E, d_best_r, cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sbh::set_error(std::string("sb_energy_noalloc: ") + cudaGetErrorString(e));
    return SB_ERR_CUDA;
  }
  return SB_OK;
}
