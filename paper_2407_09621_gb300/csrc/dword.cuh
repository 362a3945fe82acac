// Double-word FP32 arithmetic ("dd"): a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2, about 48 significant bits. On this part the FP64 pipe delivers about
// 1.25 TFLOP/s and the FP32 FMA pipe about 74.5, so FP64-vector work written with these
// operations (7-15 FP32 operations each) runs several times faster than on the FP64 pipe while
// keeping a relative error per operation near 2^-47.
//
// The building blocks are the classical error-free transformations: TwoSum (Knuth: s + e = a + b
// exactly, 6 operations) and the exact product a*b = p + fma(a, b, -p). The multiply-add a*b + c
// forms the product of the high parts exactly, adds the two cross products (their low-order product
// is below the format's precision), adds c's high part with TwoSum and folds the low-order terms into
// lo. Results are not renormalized (no Fast2Sum after each operation): TwoSum of the high parts is
// exact whatever the size of lo, the few terms a contraction sums keep lo within a few ulp of hi,
// and the join to FP64 adds hi and lo exactly; this saves 3 of 15 operations per multiply-add.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace tp {

struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dd(int v) : hi((float)v), lo(0.f) {}
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dd(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
  const dd s = dd_two_sum(a.hi, b.hi);
  return dd(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + dd(-b.hi, -b.lo); }
__device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dd(p, e);
}
// a * b + c
__device__ __forceinline__ dd fma(dd a, dd b, dd c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const dd s = dd_two_sum(p, c.hi);
  return dd(s.hi, s.lo + (e + c.lo));
}

// double -> dd with integer operations only: hi is the double's top 24 significand bits
// (truncated), lo the remaining 29 bits rounded to FP32. Magnitudes below 2^-126 become 0, those
// below 2^-74 keep hi alone (24 bits: lo would be below the FP32 normal range), and above 2^127 are
// not representable (this library's vectors stay far inside that range).
__device__ __forceinline__ dd dd_from_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);  // biased exponent
  if (e < 1023 - 126) return dd(0.f, 0.f);
  const unsigned long long mant = b & 0xfffffffffffffULL;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(mant >> 29));
  // the low 29 bits are worth m_lo * 2^(e - 1023 - 52)
  const unsigned m_lo = (unsigned)(mant & 0x1fffffffULL);
  const int se = e - 1023 - 52 + 127;  // biased FP32 exponent of 2^(e - 1075)
  const float scale = se > 0 ? __uint_as_float((unsigned)se << 23) : 0.f;
  const float lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn(m_lo) * scale));
  return dd(hi, lo);
}
// dd -> double: both parts widened exactly, one FP64 addition
__device__ __forceinline__ double dd_to_double(dd v) { return (double)v.hi + (double)v.lo; }

// host: the nearest dd of a double
inline dd dd_from_double_host(double v) {
  const float h = (float)v;
  return dd(h, (float)(v - (double)h));
}

}  // namespace tp
