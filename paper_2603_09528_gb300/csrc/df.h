// Float-pair ("double-float") arithmetic on the float32 pipe, shared by the
// mixed-precision solve and the projection: a value is hi + lo with two
// floats, operations by Knuth's TwoSum and FMA-based TwoProd, and exact
// conversions from and to float64 by integer operations (GB300's float64
// pipe runs at ~1/55 of the float32 rate and also carries the float64
// conversion instructions).
#pragma once

#include <cuda_runtime.h>

namespace tpt {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, {-y.hi, -y.lo}); }
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_from_double(double v) {
  const float h = static_cast<float>(v);
  return {h, static_cast<float>(v - static_cast<double>(h))};
}
// the rare-path conversion, kept out of line so the compiler cannot predicate
// its float64 instructions into the common path
static __device__ __noinline__ df df_from_double_slow(double v) { return df_from_double(v); }

// float64 -> float pair with integer operations only (GB300's float64 pipe,
// which also runs float64 conversions, is ~1/55 of the float32 rate): hi
// takes the leading 24 significant bits, lo the remaining 29 truncated to 24,
// so hi + lo equals v to 2^-47 relative.  Zero, |v| < 2^-47 and values beyond
// the float range go through the conversion instructions instead.
__device__ __forceinline__ df split_double_int(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned sign = static_cast<unsigned>(b >> 63) << 31;
  const int e = static_cast<int>((b >> 52) & 0x7FF);
  const int fe = e - 896;                            // float biased exponent of hi
  if (fe < 80 || fe >= 255) return df_from_double_slow(v);   // keeps lo a normal float
  const unsigned long long m = b & ((1ull << 52) - 1);
  const float hi = __uint_as_float(sign | (static_cast<unsigned>(fe) << 23) | static_cast<unsigned>(m >> 29));
  const unsigned r = static_cast<unsigned>(m & ((1u << 29) - 1));
  if (r == 0) return {hi, 0.0f};
  const int p = 31 - __clz(r);                       // leading bit of the remainder
  const int le = fe - 52 + p;                        // its float biased exponent (> 0 here)
  const unsigned frac = ((r << (31 - p)) << 1) >> 9; // bits below the leading one, 23 kept
  return {hi, __uint_as_float(sign | (static_cast<unsigned>(le) << 23) | frac)};
}

// float -> float64, exact, with integer operations (normal numbers and zero).
// Zero and subnormals map to a signed zero, infinities and NaN to the float64
// exponent 2047, all without conversion instructions.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFF;
  const unsigned long long sign = static_cast<unsigned long long>(u >> 31) << 63;
  const unsigned long long ee = (e == 0) ? 0ull : (e == 255 ? 2047ull : static_cast<unsigned long long>(e + 896));
  const unsigned long long mm = (e == 0) ? 0ull : (static_cast<unsigned long long>(u & 0x7FFFFF) << 29);
  return __longlong_as_double(static_cast<long long>(sign | (ee << 52) | mm));
}

}  // namespace tpt
