// Gather-ceiling probe (see probe.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sbd {

// grid CTAs of gather_probe_block() threads; each warp reads pairs of rows
// idx[2w + 2k warps], idx[... + 1] (row_f4 float4 each, a multiple of 32) and
// writes one partial sum to out[w] (out holds grid * block / 32 floats)
cudaError_t launch_gather_probe(const float4* a, int64_t rows, int row_f4, const int32_t* idx,
                                int64_t count, float* out, int grid, cudaStream_t s);
int gather_probe_block();
// resident CTAs per SM of the probe kernel (0 on error)
int gather_probe_blocks_per_sm();

}  // namespace sbd
