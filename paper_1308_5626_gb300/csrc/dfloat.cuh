// Double-float arithmetic on the FP32 pipe (internal).  GB300's FP64 pipe is a small
// fraction of its FP32 pipe, so the FP64-grade sums of the band fit and of the mixed form's
// restart residual are carried as unevaluated pairs hi + lo of FP32 values: an error-free
// product (Dekker, by one FMA) and Knuth's error-free two-sum keep about 48 significant bits.
// Two lanes (two rows or two grid points) go through one packed FP32x2 instruction
// (mul/fma/add/sub.rn.f32x2), the pair held in one 64-bit register.
#pragma once

#include <cstdint>

namespace psp {

__device__ __forceinline__ uint64_t f2pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2unpack(uint64_t v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2neg(uint64_t a) { return a ^ 0x8000000080000000ull; }

// x = hi + lo with hi = x rounded to the nearest FP32 (ties to even) and lo = x - hi rounded
// to FP32 (|lo| <= half an FP32 ulp of hi; hi + lo carries x to about 2^-48 relative), from
// the bits of x with integer operations only.  For 2^-126 <= |x| < 2^128 the split follows
// from the IEEE 754 binary64 layout: hi keeps the sign, the exponent rebiased from 1023 to
// 127 and the top 23 stored mantissa bits, rounded on the 29 dropped bits; x - hi is the
// signed remainder of those 29 bits (at most 2^28 in magnitude) times 2^(e - 1075), e the
// biased binary64 exponent.  Outside that range (zero, FP32-subnormal or overflowing
// magnitudes, inf, NaN) hi is the FP64 to FP32 conversion and lo = 0.
__device__ __forceinline__ void split_double(double x, float &hi, float &lo) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const uint32_t sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  const int ef = e - 896;                 // FP32 biased exponent of x: e - 1023 + 127
  if (ef < 1 || ef > 254) {
    hi = (float)x;
    lo = 0.0f;
    return;
  }
  const uint32_t mt = ((hw & 0xfffffu) << 3) | (lw >> 29);   // top 23 stored mantissa bits
  const uint32_t rest = lw & 0x1fffffffu;                     // the 29 dropped bits
  const uint32_t up = (rest > 0x10000000u) | ((rest == 0x10000000u) & mt & 1u);
  hi = __uint_as_float(sign | ((((uint32_t)ef << 23) | mt) + up));   // a carry moves into the exponent
  const int es = e - 948;                 // FP32 biased exponent of 2^(e - 1075)
  if (es < 1) {
    lo = 0.0f;                            // |x - hi| < 2^-98 |x|: below the pair's resolution
    return;
  }
  const float l = (float)((int)rest - (int)(up << 29)) * __uint_as_float((uint32_t)es << 23);
  lo = sign ? -l : l;
}

}  // namespace psp
