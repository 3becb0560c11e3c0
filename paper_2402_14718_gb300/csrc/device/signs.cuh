// Signs of positions, as used by the dSB coupling product (Eq. 10 takes
// sgn(x_j)), without the slow int -> float conversion.
#pragma once
#include <stdint.h>

namespace sbd {

// sgn(x) with sgn(0) = 0, as a float, in compares and selects only.
__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// A sign stored as one byte, biased by 128: 127, 128 or 129 for -1, 0, +1.
__device__ __forceinline__ uint32_t sign_byte(float x) {
  return 128u + (x > 0.f ? 1u : 0u) - (x < 0.f ? 1u : 0u);
}

// Byte k of w (a biased sign) as the float -1, 0 or +1, exactly: the byte is
// placed in the low mantissa byte of 2^23 (bits 0x4B000000), which then reads
// 2^23 + byte, and 2^23 + 128 is subtracted. One byte permute and one add,
// both at full rate.
__device__ __forceinline__ float sign_of_byte(uint32_t w, int k) {
  return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7650u | (uint32_t)k)) - 8388736.0f;
}

}  // namespace sbd
