// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
// written from the published definition: 10 rounds; each round multiplies
// counter words 0 and 2 by fixed 32-bit constants, and the new counter is
// (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key advances by two Weyl
// constants between rounds. Usable from host C++ and CUDA device code.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SB_HD __host__ __device__ __forceinline__
#else
#define SB_HD inline
#endif

namespace sbk {

enum : uint32_t { kPurposeTrack = 1, kPurposeNoise = 2, kPurposeInit = 3 };

struct U32x4 {
  uint32_t v[4];
};

SB_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

SB_HD U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                          uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += W0;
      k1 += W1;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(M0, c0, &hi0, &lo0);
    mulhilo32(M1, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  U32x4 r;
  r.v[0] = c0;
  r.v[1] = c1;
  r.v[2] = c2;
  r.v[3] = c3;
  return r;
}

// U[0,1) from 64 bits (lo | hi << 32): top 53 bits times 2^-53.
SB_HD double uniform01(uint32_t lo, uint32_t hi) {
  uint64_t u = (uint64_t)lo | ((uint64_t)hi << 32);
  return (double)(u >> 11) * 0x1.0p-53;
}

// SB initial value in U(-0.01, 0.01): v = (w >> 8) - 2^23, x = fp32(v) * (fp32(0.01) * 2^-23).
SB_HD float init_value(uint32_t w) {
  int32_t v = (int32_t)(w >> 8) - (1 << 23);
  const float scale = 0.01f * 0x1.0p-23f;
  return (float)v * scale;
}

}  // namespace sbk
