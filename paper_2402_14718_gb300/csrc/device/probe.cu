// Gather-ceiling probe: the rate at which the SMs can read whole rows of an
// array at random row indices, the access pattern of the coupling product
// (each neighbour of a row brings that neighbour's replica row). Each warp
// reads its rows with 16-byte loads per lane, two rows in flight, the way the
// row-group step kernel does, and folds them into a sum that it writes out (so
// that no load is dropped). It runs on its own: the measured bytes per second
// are an on-chip ceiling for the step's neighbour reads, beside the HBM one.
#include <cuda_runtime.h>
#include <stdint.h>

#include "probe.cuh"

namespace sbd {
namespace {

constexpr int kProbeBlock = 128;

// rows of row_f4 float4 (row_f4 a multiple of 32: whole 512-byte chunks per
// warp); idx: `count` row indices, each < rows; out: one float per warp
__global__ void __launch_bounds__(kProbeBlock) k_gather_probe(const float4* a, int64_t rows,
                                                              int row_f4, const int32_t* idx,
                                                              int64_t count, float* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kProbeBlock + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * kProbeBlock) >> 5;
  const int chunks = row_f4 / 32;
  float s = 0.f;
  int64_t i = warp * 2;
  for (; i + 1 < count; i += warps * 2) {
    const int64_t r0 = __ldg(idx + i), r1 = __ldg(idx + i + 1);
    if (r0 < 0 || r0 >= rows || r1 < 0 || r1 >= rows) continue;
    for (int c = 0; c < chunks; ++c) {
      const float4 u = __ldg(a + r0 * row_f4 + c * 32 + lane);
      const float4 v = __ldg(a + r1 * row_f4 + c * 32 + lane);
      s += (u.x + u.y) + (u.z + u.w) + (v.x + v.y) + (v.z + v.w);
    }
  }
  if (lane == 0) out[warp] = s;
}

}  // namespace

cudaError_t launch_gather_probe(const float4* a, int64_t rows, int row_f4, const int32_t* idx,
                                int64_t count, float* out, int grid, cudaStream_t s) {
  if (row_f4 <= 0 || row_f4 % 32 != 0 || rows <= 0 || count < 2 || grid <= 0)
    return cudaErrorInvalidValue;
  k_gather_probe<<<grid, kProbeBlock, 0, s>>>(a, rows, row_f4, idx, count, out);
  return cudaGetLastError();
}

int gather_probe_block() { return kProbeBlock; }

int gather_probe_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_probe, kProbeBlock, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace sbd
