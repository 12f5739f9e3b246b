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

// The same split of x 2^-shift (shift an exponent, so the scaling is exact); ok becomes false
// when x 2^-shift is neither zero nor inside FP32's normal range (hi and lo are then not the
// split and the caller takes another path).
__device__ __forceinline__ void split_double_scaled(double x, int shift, float &hi, float &lo, bool &ok) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const uint32_t sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  if (e == 0 && (hw & 0xfffffu) == 0 && lw == 0) {   // +-0
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  const int ef = e - 896 - shift;
  if (e == 0 || e == 0x7ff || ef < 1 || ef > 254) {
    hi = 0.0f;
    lo = 0.0f;
    ok = false;
    return;
  }
  const uint32_t mt = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const uint32_t rest = lw & 0x1fffffffu;
  const uint32_t up = (rest > 0x10000000u) | ((rest == 0x10000000u) & mt & 1u);
  const uint32_t hb = (((uint32_t)ef << 23) | mt) + up;
  if ((hb >> 23) > 254u) {   // rounded up past FP32's range
    hi = 0.0f;
    lo = 0.0f;
    ok = false;
    return;
  }
  hi = __uint_as_float(sign | hb);
  const int es = ef - 52;    // FP32 biased exponent of 2^(e - 1075 - shift)
  if (es < 1) {
    lo = 0.0f;
    return;
  }
  const float l = (float)((int)rest - (int)(up << 29)) * __uint_as_float((uint32_t)es << 23);
  lo = sign ? -l : l;
}

// Scalar double-float values (hi + lo, |lo| at most half an FP32 ulp of hi) and the
// operations of the band fit's row solves.  The _rn intrinsics keep the compiler from
// contracting an error-free step into an FMA.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ double df_value(DF a) { return (double)a.hi + (double)a.lo; }
// s + t renormalised (fast two-sum: |s| >= |t|)
__device__ __forceinline__ DF df_norm(float s, float t) {
  const float h = __fadd_rn(s, t);
  DF r;
  r.hi = h;
  r.lo = __fsub_rn(t, __fsub_rn(h, s));
  return r;
}
// a - b c: the product exactly (b_hi c_hi = p + e by one FMA) but for the b_lo c_lo term, then
// Knuth's two-sum of a_hi and -p, the low parts after it
__device__ __forceinline__ DF df_fms(DF a, DF b, DF c) {
  const float p = __fmul_rn(b.hi, c.hi);
  float e = fmaf(b.hi, c.hi, -p);
  e = fmaf(b.hi, c.lo, e);
  e = fmaf(b.lo, c.hi, e);
  const float s = __fsub_rn(a.hi, p);
  const float v = __fsub_rn(s, a.hi);
  const float err = __fsub_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fadd_rn(p, v));
  return df_norm(s, __fadd_rn(err, __fsub_rn(a.lo, e)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_norm(p, e);
}
// 1 / sqrt(d), d > 0 in FP32's normal range: the FP32 estimate and two Newton steps
// r <- r + r (1 - d r^2) / 2 with d r^2 in double-float (each step squares the relative error,
// from the estimate's ~2^-22 to below the pair's resolution)
__device__ __forceinline__ DF df_rsqrt(DF d) {
  DF r;
  r.hi = rsqrtf(d.hi);
  r.lo = 0.0f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const DF h = df_mul(df_mul(d, r), r);               // 1 + O(error): 1 - h_hi is exact
    const float t = __fsub_rn(__fsub_rn(1.0f, h.hi), h.lo);
    const float c = __fmul_rn(__fmul_rn(r.hi, t), 0.5f);
    r = df_norm(r.hi, __fadd_rn(r.lo, c));
  }
  return r;
}

}  // namespace psp
