// Signs of positions, as used by the dSB coupling product (Eq. 10 takes
// sgn(x_j)), without the slow int -> float conversion.
#pragma once
#include <stdint.h>

namespace sbd {

// sgn(x) with sgn(0) = 0, as a float, in compares and selects only.
__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// A sign stored as one byte: 0x3C, 0xBC or 0x00 for x > 0, x < 0 and x = 0.
// Placed as the top byte of an FP32 word (the other bytes zero) it reads
// +-2^-7 (or +0).
__device__ __forceinline__ uint32_t sign_byte(float x) {
  return x > 0.f ? 0x3Cu : (x < 0.f ? 0xBCu : 0u);
}

// The FP32 reading of a sign byte is sgn * 2^-7, so an FP32 coupling product
// takes it with the weight scaled by 2^7: fma(2^7 J, 2^-7 sgn, acc) equals
// fma(J, sgn, acc) bit for bit (2^7 J is exact for |J| < 2^120, and the
// product is exactly J sgn, leaving the one rounding of the sum).
constexpr float kSignScale = 128.f;

// Byte k of w as the float sgn * 2^-7, in one byte permute: the byte goes to
// the top of a word whose other bytes are zero.
__device__ __forceinline__ float scaled_sign_of_byte(uint32_t w, int k) {
  return __int_as_float((int)__byte_perm(w, 0u, 0x0444u | ((uint32_t)k << 12)));
}

// Ask for the 128-byte line holding p to be brought into L2 (no register is
// written; a later load of it then hits L2 instead of waiting on HBM).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// True when the two float4 differ in any bit (a state value that did not
// change need not be written back where it is updated in place).
__device__ __forceinline__ bool bits_differ(const float4& a, const float4& b) {
  return (__float_as_uint(a.x) ^ __float_as_uint(b.x)) | (__float_as_uint(a.y) ^ __float_as_uint(b.y)) |
         (__float_as_uint(a.z) ^ __float_as_uint(b.z)) | (__float_as_uint(a.w) ^ __float_as_uint(b.w));
}

}  // namespace sbd
