// vmath.cuh -- the operations the face arithmetic is written with, per value type: double (FP64
// path) and float (mixed path), with explicit fused multiply-adds; and integer-pipe f32 <-> f64
// conversions.
#pragma once
#include <cuda_runtime.h>

namespace gbcfd {

// the operations the generic code uses, per value type
template <typename V> struct VM;

template <> struct VM<double> {
  using S = double;
  static __device__ __forceinline__ double c(double s) { return s; }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ double rsqrt(double a) { return ::rsqrt(a); }
  static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
  static __device__ __forceinline__ double ab(double a) { return fabs(a); }
  static __device__ __forceinline__ double mn(double a, double b) { return fmin(a, b); }
  static __device__ __forceinline__ double csign(double q, double x) { return copysign(q, x); }
  // a < b ? x : y
  static __device__ __forceinline__ double lt(double a, double b, double x, double y) { return a < b ? x : y; }
  static __device__ __forceinline__ double pos(double a, double x, double y) { return a > 0.0 ? x : y; }
};

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
