// FP64 <-> FP32 conversions on the integer pipe, from the IEEE-754 bit layouts.
//
// On GB300 a cvt between FP64 and FP32 issues on the FP64 pipe, as slowly as a DFMA, so the
// mixed-precision Gram-Schmidt sweeps convert with integer instructions instead:
//   to_f32  truncates the significand to 24 bits (relative error below 2^-23), flushes magnitudes
//           under 2^-126 to zero, sends finite values of 2^128 and above to +-Inf, and keeps Inf
//           and NaN (a NaN stays a quiet NaN whatever its payload);
//   to_f64  is exact for normal floats, Inf and NaN, and flushes subnormal floats to zero.
// The same functions compile for the host (bit casts through memcpy), so their special cases are
// tested on the CPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace dg {

__host__ __device__ __forceinline__ uint64_t bits_of(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ float float_of(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
__host__ __device__ __forceinline__ uint32_t bits_of(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ double double_of(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t b = ((uint64_t)hi << 32) | lo;
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}

__host__ __device__ __forceinline__ float to_f32(double d) {
  const uint64_t b = bits_of(d);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t e = (hi >> 20) & 0x7ffu;
  const uint32_t frac = ((hi & 0xfffffu) << 3) | (lo >> 29);      // top 23 significand bits
  const bool nan = e == 0x7ffu && (((hi & 0xfffffu) | lo) != 0u);
  // exponent: 0 below 2^-126, 255 for Inf, NaN and finite overflow, else rebiased
  const uint32_t ef = e < 897u ? 0u : (e > 1150u ? 255u : e - 896u);
  const uint32_t m = nan ? (frac | 0x400000u) : ((ef == 0u || ef == 255u) ? 0u : frac);
  return float_of((hi & 0x80000000u) | (ef << 23) | m);
}

__host__ __device__ __forceinline__ double to_f64(float f) {
  const uint32_t b = bits_of(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t ed = e == 0u ? 0u : (e == 255u ? 0x7ffu : e + 896u);
  const uint32_t hi = (b & 0x80000000u) | (ed << 20) | (e ? ((b & 0x7fffffu) >> 3) : 0u);
  return double_of(hi, e ? b << 29 : 0u);
}

}  // namespace dg
