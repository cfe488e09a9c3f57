// FP64 -> FP32 conversion in integer arithmetic, for the mixed-precision
// contraction kernels.  B300 executes FP64 instructions (conversions
// included) at a small fraction of its FP32 and integer rates, and operand
// tiles stored in FP64 are converted element by element on their way to an
// FP32 or TF32 multiplication, so the conversion is done on the bit pattern:
// the 23 leading mantissa bits, rounded on the next bit (ties away from
// zero), exponent rebiased; results in the FP32 subnormal range keep the bits
// that fit, results above the largest FP32 number become infinity, NaN stays
// NaN.
#pragma once
#include <cstdint>

namespace sgtn {

__device__ __forceinline__ float f64_to_f32_int(double v) {
  const uint32_t h = (uint32_t)__double2hiint(v), l = (uint32_t)__double2loint(v);
  const uint32_t sign = h & 0x80000000u;
  const int e = int((h >> 20) & 0x7FFu);
  const uint32_t m = ((h & 0xFFFFFu) << 3) | (l >> 29);   // 23 mantissa bits
  const uint32_t r = (l >> 28) & 1u;                      // first dropped bit
  const int e32 = e - (1023 - 127);
  uint32_t f;
  if (e == 0x7FF) f = ((h & 0xFFFFFu) | l) ? 0x7FC00000u : 0x7F800000u;
  else if (e32 <= 0) {
    // subnormal: the 24-bit significand shifted right by 1 - e32, rounded on
    // the last bit shifted out (0 when nothing is left)
    const int sh = 1 - e32;
    if (sh > 24) {
      f = 0u;
    } else {
      const uint32_t sig = (1u << 23) | m;
      f = (sig >> sh) + ((sig >> (sh - 1)) & 1u);
    }
  }
  else if (e32 >= 255) f = 0x7F800000u;
  else f = ((uint32_t)e32 << 23) + m + r;   // a mantissa carry moves into the exponent
  if (f > 0x7F800000u && e != 0x7FF) f = 0x7F800000u;
  return __uint_as_float(f | sign);
}

}  // namespace sgtn
