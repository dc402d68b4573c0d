// Complex64 helpers without float<->double conversion instructions.
//
// The complex64 form computes two values in FP64 (Sec. III bookkeeping):
//   prob(re, im) = fma(double(re), double(re), double(im) * double(im))
//   scaled(x, s) = float(double(x) * s)
// On B300 the float<->double conversion instructions, not the FP64 multiply
// and fma, limit these (measured: about half the throughput of the forms
// below).  Here the widening float -> double (exact) and the narrowing
// double -> float (IEEE 754 round to nearest, ties to even, with the
// subnormal grid and overflow) are done by bit manipulation of the
// significand and exponent, and the multiply and fma stay FP64 instructions,
// so the results are the same bits; sv_selftest checks that on the device.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace sv {

// Significand and exponent of |x| for a finite float: |x| = m * 2^e.
__device__ __forceinline__ void f32_split(float x, uint32_t* m, int* e) {
  const uint32_t b = __float_as_uint(x) & 0x7fffffffu;
  const uint32_t ex = b >> 23;
  if (ex == 0) {
    *m = b;  // zero or subnormal
    *e = -149;
  } else {
    *m = (b & 0x7fffffu) | 0x800000u;
    *e = (int)ex - 150;
  }
}

// f32_split with subnormals normalised: m in [2^23, 2^24) unless x == 0.
__device__ __forceinline__ void f32_split_norm(float x, uint32_t* m, int* e) {
  f32_split(x, m, e);
  if (*m && *m < 0x800000u) {
    const int k = __clz(*m) - 8;  // bring the leading bit to position 23
    *m <<= k;
    *e -= k;
  }
}

// Exact float -> double by bit manipulation (no conversion instruction).
// Normal floats (the usual case) move their exponent from bias 127 to 1023
// and their significand up by 29 bits in one add and one shift; zeros and
// subnormals take the general path below.
__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const uint32_t b = __float_as_uint(x);
  if (((b >> 23) & 0xffu) != 0u && ((b >> 23) & 0xffu) != 0xffu)
    return __longlong_as_double((long long)(((uint64_t)(b & 0x80000000u) << 32) |
                                            (((uint64_t)(b & 0x7fffffffu) + (896ull << 23)) << 29)));
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  uint32_t m;
  int e;
  f32_split_norm(x, &m, &e);
  if (m == 0) return __longlong_as_double((long long)sign);
  // |x| = m * 2^e with m in [2^23, 2^24): double exponent e + 23
  return __longlong_as_double(
      (long long)(sign | ((uint64_t)(e + 23 + 1023) << 52) | (((uint64_t)m << 29) & ((1ull << 52) - 1))));
}

// Round a finite double to the nearest float, ties to even, by bit
// manipulation (normal, subnormal and overflowing results).
__device__ __forceinline__ float f64_to_f32_rn_bits(double v) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int E = (int)((b >> 52) & 0x7ffu) - 1023;
  if (((b >> 52) & 0x7ffu) == 0) return __uint_as_float(sign);  // zero or double subnormal: below float range
  const uint64_t m53 = (b & ((1ull << 52) - 1)) | (1ull << 52);
  int sh = 29;
  if (E < -126) sh = 29 + (-126 - E);
  if (sh >= 64) return __uint_as_float(sign);
  uint64_t m = m53 >> sh;
  const uint64_t rem = m53 & ((1ull << sh) - 1ull);
  const uint64_t half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (m & 1ull))) ++m;
  if (E < -126) return __uint_as_float(sign | (uint32_t)m);  // subnormal grid (2^23 = smallest normal)
  int ee = E;
  if (m >> 24) {
    m >>= 1;
    ++ee;
  }
  if (ee > 127) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((uint32_t)(ee + 127) << 23) | ((uint32_t)m & 0x7fffffu));
}

// float(double(x) * s) with the multiply on the FP64 pipe and both
// conversions as integer bit manipulation.
__device__ __forceinline__ float scaled_f32_mul(float x, double s) {
  return f64_to_f32_rn_bits(__dmul_rn(f32_to_f64_bits(x), s));
}

// Probability bits of an amplitude in its own precision: the FP64 formula
// for complex128, the integer-pipe equivalent for complex64.
__device__ __forceinline__ uint64_t amp_prob_bits(double re, double im) {
  return (uint64_t)__double_as_longlong(prob_of(re, im));
}
__device__ __forceinline__ uint64_t amp_prob_bits(float re, float im) {
  return (uint64_t)__double_as_longlong(prob_of(f32_to_f64_bits(re), f32_to_f64_bits(im)));
}
__device__ __forceinline__ uint64_t amp_prob_bits(double2 a) { return amp_prob_bits(a.x, a.y); }
__device__ __forceinline__ uint64_t amp_prob_bits(float2 a) { return amp_prob_bits(a.x, a.y); }

// Renormalised amplitude: x * s in FP64 for complex128, float(double(x) * s)
// for complex64.
__device__ __forceinline__ double2 amp_scaled(double2 a, double s) {
  return make_double2(__dmul_rn(a.x, s), __dmul_rn(a.y, s));
}
__device__ __forceinline__ float2 amp_scaled(float2 a, double s) {
  return make_float2(scaled_f32_mul(a.x, s), scaled_f32_mul(a.y, s));
}

}  // namespace sv
