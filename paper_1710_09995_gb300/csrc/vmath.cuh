// vmath.cuh -- the operations the face arithmetic is written with, per value type: double (FP64
// path) and float (mixed path), with explicit fused multiply-adds; and integer-pipe f32 <-> f64
// conversions.
#pragma once
#include <cuda_runtime.h>

namespace gbcfd {

// the operations the generic code uses, per value type
template <typename V> struct VM;

// The FP64 path is bound by the FP64 pipe (this part issues one FP64 operation per 64 FP32
// ones), while its integer pipe idles: comparisons whose operands are known to be non-negative
// run there on the bit patterns (for non-negative IEEE doubles the order of the values is the
// order of their bit patterns as unsigned integers), and the reciprocal is the hardware's
// estimate refined by Newton's method instead of an IEEE division.
template <> struct VM<double> {
  using S = double;
  static __device__ __forceinline__ double c(double s) { return s; }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ double rsqrt(double a) { return ::rsqrt(a); }
  // 1/a for positive finite a: the estimate r of rcp.approx.ftz.f64 (relative error e0 about
  // 2^-22) and one third-order Newton step r (1 + e + e^2), e = 1 - a r, whose relative error is
  // e0^3: three FMAs.  Within an ulp or two of the correctly rounded quotient, not always equal to
  // it.  a = 0 gives NaN (callers select such values away).
  static __device__ __forceinline__ double rcp(double a) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(a));
    const double e = ::fma(-a, r, 1.0);
    return ::fma(r, ::fma(e, e, e), r);
  }
  static __device__ __forceinline__ double ab(double a) { return fabs(a); }
  static __device__ __forceinline__ double mn(double a, double b) { return fmin(a, b); }
  static __device__ __forceinline__ double csign(double q, double x) { return copysign(q, x); }
  // a < b ? x : y, for non-negative a and b: compared as bit patterns on the integer pipe
  static __device__ __forceinline__ double lt(double a, double b, double x, double y) {
    return (unsigned long long)__double_as_longlong(a) < (unsigned long long)__double_as_longlong(b) ? x : y;
  }
  // a > 0 ? x : y, for non-negative a (its bit pattern is non-zero)
  static __device__ __forceinline__ double pos(double a, double x, double y) {
    return __double_as_longlong(a) != 0ll ? x : y;
  }
};

// Half the minmod slope of the differences a and b in doubles, on the integer pipe: zero when
// their signs differ or either is zero, else the smaller magnitude (compared as bit patterns)
// halved by lowering its exponent by one, with the common sign.  Exact for every magnitude of
// at least 2^-1021; smaller ones (subnormal halves) give zero.
__device__ __forceinline__ double half_minmod_f64(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const unsigned long long ma = (unsigned long long)ia & 0x7fffffffffffffffull;
  const unsigned long long mb = (unsigned long long)ib & 0x7fffffffffffffffull;
  const unsigned long long m = ma < mb ? ma : mb;
  const unsigned long long h = m >= (2ull << 52) ? m - (1ull << 52) : 0ull;
  const unsigned long long sgn = (unsigned long long)ia & 0x8000000000000000ull;
  return __longlong_as_double((ia ^ ib) >= 0 ? (long long)(h | sgn) : 0ll);
}

template <> struct VM<float> {
  using S = float;
  static __device__ __forceinline__ float c(float s) { return s; }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ float rsqrt(float a) { return rsqrtf(a); }
  static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.0f, a); }
  static __device__ __forceinline__ float ab(float a) { return fabsf(a); }
  static __device__ __forceinline__ float mn(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float csign(float q, float x) { return copysignf(q, x); }
  static __device__ __forceinline__ float lt(float a, float b, float x, float y) { return a < b ? x : y; }
  static __device__ __forceinline__ float pos(float a, float x, float y) { return a > 0.f ? x : y; }
};

// f32 <-> f64 conversions with integer bit operations, so they issue on the integer pipe instead
// of the slow FP64 pipe (where F2F conversions run on this part).  Exact / round-to-nearest-even
// like the hardware conversions for finite normal values; zero and subnormal inputs become a
// signed zero, non-finite inputs stay non-finite.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned sign = b & 0x80000000u;
  unsigned hi, lo;
  if (e == 0u) {
    hi = sign; lo = 0u;
  } else if (e == 0xffu) {
    hi = sign | 0x7ff00000u | ((b & 0x7fffffu) >> 3); lo = b << 29;
  } else {
    hi = sign | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    lo = b << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffull) - 1023 + 127;
  if (((b >> 52) & 0x7ffull) == 0x7ffull)  // inf or nan
    return __uint_as_float(sign | 0x7f800000u | (unsigned)((b & 0xfffffffffffffull) != 0ull));
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long m = b & 0xfffffffffffffull;  // 52 bits
  unsigned r = ((unsigned)e << 23) | (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1fffffffull), halfway = 0x10000000u;
  r += (rem > halfway || (rem == halfway && (r & 1u))) ? 1u : 0u;  // carry may step the exponent
  if (r >= 0x7f800000u) r = 0x7f800000u;
  return __uint_as_float(sign | r);
}

}  // namespace gbcfd
