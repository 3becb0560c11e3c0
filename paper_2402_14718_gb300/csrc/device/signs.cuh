// Signs of positions, as used by the dSB coupling product (Eq. 10 takes
// sgn(x_j)), without the slow int -> float conversion.
#pragma once
#include <stdint.h>

namespace sbd {

// sgn(x) with sgn(0) = 0, as a float, in compares and selects only.
__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// A sign stored as one byte: the top byte of the float +0.5 (0x3F), -0.5
// (0xBF) or +0 (0x00), for x > 0, x < 0 and x = 0.
__device__ __forceinline__ uint32_t sign_byte(float x) {
  return x > 0.f ? 0x3Fu : (x < 0.f ? 0xBFu : 0u);
}

// Byte k of w as the float sgn / 2 (+0.5, -0.5 or +0) in one byte permute: the
// byte goes to the top of a word whose other bytes are zero. A coupling
// product takes it with the doubled weight: fma(2 J, sgn / 2, acc) equals
// fma(J, sgn, acc) bit for bit, since 2 J is exact (|J| < 2^127) and the
// product 2 J * sgn / 2 = J sgn is exact, leaving the one rounding of the sum.
__device__ __forceinline__ float half_sign_of_byte(uint32_t w, int k) {
  return __int_as_float((int)__byte_perm(w, 0u, 0x0444u | ((uint32_t)k << 12)));
}

}  // namespace sbd
