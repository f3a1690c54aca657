// dd.cuh -- double-float arithmetic: a real number held as the unevaluated sum hi + lo of two
// floats (|lo| <= ulp(hi) / 2), about 48 significant bits, computed on the FP32 pipes.
//
// On this part the FP64 pipe runs at 1/64 of the FP32 rate, so the transforms of the mixed
// path's potential build (the density and its gradients, where the GGA functionals need far more
// than FP32's 24 bits at low density) use this representation instead of FP64.  The operations
// are the classical error-free transformations: Knuth's TwoSum for a sum with its rounding
// error, Dekker's FastTwoSum for renormalisation (|a| >= |b|), and the product with its exact
// rounding error from one fused multiply-add.  Addition follows the accurate (IEEE-style)
// double-float sum: both hi and lo parts summed with their errors, then renormalised twice.
// Intrinsics with explicit rounding keep the compiler from contracting or reordering them.
#pragma once

#include "common.cuh"

namespace fde {

struct dd {
  float hi, lo;
  __host__ __device__ __forceinline__ dd() {}
  __host__ __device__ __forceinline__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // Exact small integers and literal constants (the split folds at compile time).
  __host__ __device__ __forceinline__ constexpr dd(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ __forceinline__ constexpr dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ dd(long double v) : hi((float)v), lo((float)(v - (long double)(float)v)) {}
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return dd(s, e);
}
__device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return dd(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  const dd t = dd_two_sum(a.lo, b.lo);
  s = dd_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return dd_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_fast_two_sum(p, e);
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__device__ __forceinline__ dd& operator-=(dd& a, dd b) { return a = a - b; }
__device__ __forceinline__ dd& operator*=(dd& a, dd b) { return a = a * b; }

// Conversions at the boundary of a transform (FP64 grids in global memory).  The FP64 pipe
// runs at 1/64 of the FP32 rate here, so the split and the join work on the bit patterns with
// integer and FP32 instructions.  The split equals the FP64-based one for 2^-70 <= |v| < 2^127;
// below 2^-70 (the vacuum tails of a density, 70 binary orders under its peak) it keeps the
// rounded high part alone (or nothing below FP32's normal range), an absolute error under
// 2^-94, and huge values take the FP64 conversions.
__device__ __forceinline__ dd dd_from_double_fp64(double v) {
  const float h = __double2float_rn(v);
  return dd(h, __double2float_rn(v - (double)h));
}
// v = (-1)^s 2^e (1 + m 2^-52): hi keeps the top 23 mantissa bits rounded to nearest even (a
// carry out of the mantissa correctly increments the exponent field), and v - hi, which is
// exactly the remaining bits minus the rounding increment times 2^(e - 52), is rounded to a
// float by the integer-to-float conversion and scaled by an exact power of two.
__device__ __forceinline__ dd dd_from_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e > 126) return dd_from_double_fp64(v);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  if (e < -126) return dd(__uint_as_float(sign), 0.0f);
  const unsigned int mh = (unsigned int)((b >> 29) & 0x7FFFFFu);
  const unsigned int rem = (unsigned int)(b & 0x1FFFFFFFu);
  const unsigned int up = (rem > 0x10000000u || (rem == 0x10000000u && (mh & 1u))) ? 1u : 0u;
  const float hi = __uint_as_float(sign | ((((unsigned int)(e + 127)) << 23) + mh + up));
  if (e < -70) return dd(hi, 0.0f);
  const int diff = (int)rem - (up ? 0x20000000 : 0);
  float lo = __int2float_rn(diff) * __uint_as_float((unsigned int)(e - 52 + 127) << 23);
  if (sign) lo = -lo;
  return dd(hi, lo);
}
// double -> float rounded to nearest even on the bit pattern (the high part of the split);
// values below FP32's normal range become zero, huge ones take the FP64 conversion.
__device__ __forceinline__ float float_of_double_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e > 126) return __double2float_rn(v);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  if (e < -126) return __uint_as_float(sign);
  const unsigned int mh = (unsigned int)((b >> 29) & 0x7FFFFFu);
  const unsigned int rem = (unsigned int)(b & 0x1FFFFFFFu);
  const unsigned int up = (rem > 0x10000000u || (rem == 0x10000000u && (mh & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | ((((unsigned int)(e + 127)) << 23) + mh + up));
}
// Exact float -> double on the bit pattern (normal floats and zero), else the FP64 conversion.
__device__ __forceinline__ double float_to_double_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ef = (u >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  if ((u << 1) == 0u) return __longlong_as_double((long long)s);
  if (ef == 0u || ef == 255u) return (double)f;
  return __longlong_as_double((long long)(s | ((unsigned long long)(ef - 127u + 1023u) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ double dd_to_double(dd v) { return float_to_double_bits(v.hi) + float_to_double_bits(v.lo); }

struct __align__(16) ddc {
  dd x, y;
};
template <> struct cx<dd> { using t = ddc; };

}  // namespace fde
