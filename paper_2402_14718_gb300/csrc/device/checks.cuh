// Index checks of the bounds-checked build (every .cu compiled with
// -DSB_CHECKED=1; the release build compiles them away).
//
// A checked index that falls outside its array is recorded in the module's
// error word -- the first one only: site code in the high 32 bits, the index
// in the low 32 -- and replaced by 0, so the access stays inside the array
// and nothing traps. A row-pointer pair outside [0, nnz] or decreasing is
// recorded the same way and read as an empty row. The host reads and clears
// the words of every module with sb_check_bounds.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef SB_CHECKED
#define SB_CHECKED 0
#endif

namespace sbd {

// what a recorded index was (the high word of an error word)
enum CheckSite : uint32_t {
  kChkCol = 1,      // a CSR column (neighbour row) of a step or energy kernel
  kChkRowptr = 2,   // a row-pointer pair (the row's end is recorded)
  kChkURow = 3,     // a U row of the factored product
  kChkMember = 4,   // a group member row of the factored group sums
  kChkEntry = 5,    // a column of a row-group union entry
};

#if SB_CHECKED
// one word per module (each .cu is its own module: the library is built
// without relocatable device code)
static __device__ unsigned long long g_chk_word;

__device__ __forceinline__ void chk_record(uint32_t site, uint32_t v) {
  atomicCAS(&g_chk_word, 0ull, ((unsigned long long)site << 32) | v);
}
// i if 0 <= i < bound, else 0 (recorded)
__device__ __forceinline__ int chk_idx(int i, int bound, uint32_t site) {
  if ((unsigned)i < (unsigned)bound) return i;
  chk_record(site, (uint32_t)i);
  return 0;
}
// a row's pointer pair: 0 <= p0 <= p1 <= nnz, else an empty row (recorded)
__device__ __forceinline__ void chk_rows(int& p0, int& p1, long long nnz) {
  if (p0 >= 0 && p0 <= p1 && (long long)p1 <= nnz) return;
  chk_record(kChkRowptr, (uint32_t)p1);
  p0 = p1 = 0;
}
// Defines `cudaError_t fn(unsigned long long* w)`: the module's word into *w,
// then cleared (synchronous copies on the current device).
#define SB_CHECK_READER(fn)                                                    \
  cudaError_t fn(unsigned long long* w) {                                      \
    cudaError_t e_ = cudaMemcpyFromSymbol(w, g_chk_word, sizeof(*w));          \
    if (e_ != cudaSuccess) return e_;                                          \
    const unsigned long long z_ = 0;                                           \
    return cudaMemcpyToSymbol(g_chk_word, &z_, sizeof(z_));                    \
  }
#else
__device__ __forceinline__ int chk_idx(int i, int, uint32_t) { return i; }
__device__ __forceinline__ void chk_rows(int&, int&, long long) {}
#define SB_CHECK_READER(fn)                                                    \
  cudaError_t fn(unsigned long long* w) {                                      \
    *w = 0;                                                                    \
    return cudaSuccess;                                                        \
  }
#endif

// one reader per module that holds checked kernels
cudaError_t chk_read_kernels(unsigned long long* w);
cudaError_t chk_read_factor(unsigned long long* w);
cudaError_t chk_read_rw(unsigned long long* w);

}  // namespace sbd
