// Conversions between binary32 and binary64 by integer operations.
//
// On GB300 a conversion instruction between the two formats runs on the FP64
// pipe, which is narrow (one warp instruction holds a sub-partition's FP64 unit
// for tens of cycles).  Kernels that compute in FP32 or double-float but convert
// a few values per thread (Bloch phases, FP64 storage read as float, FP32
// multigrid results added to FP64 iterates) were bound by those conversions.
// The functions below give the results of the IEEE conversions from the
// binary formats alone: binary32 -> binary64 is exact; binary64 -> binary32
// rounds to nearest with ties to even, produces subnormals, overflows to
// infinity and maps NaN to a quiet NaN.  They compile for host and device, so
// the host test can compare them with the compiler's conversions.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace pbs {

__host__ __device__ __forceinline__ uint32_t bits_of(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ float float_of(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}
__host__ __device__ __forceinline__ uint64_t bits_of(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  std::memcpy(&u, &d, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double double_of(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
#endif
}
__host__ __device__ __forceinline__ int clz32(uint32_t x) {  // x != 0
#ifdef __CUDA_ARCH__
  return __clz(x);
#else
  return __builtin_clz(x);
#endif
}

// binary32 -> binary64 (exact): the exponent is rebiased (127 -> 1023) and the 23
// fraction bits move to the top of the 52; a subnormal m 2^-149 is normalised first.
__host__ __device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = bits_of(f);
  const uint64_t s = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (e == 0xFFu) return double_of(s | 0x7FF0000000000000ull | ((uint64_t)m << 29) | (m ? (1ull << 51) : 0ull));
  if (e != 0u) return double_of(s | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29));
  if (m == 0u) return double_of(s);
  const int z = clz32(m) - 8;  // shift that brings the leading bit to position 23
  return double_of(s | ((uint64_t)(897 - z) << 52) | ((uint64_t)((m << z) & 0x7FFFFFu) << 29));
}

// binary64 -> binary32, round to nearest, ties to even.
__host__ __device__ __forceinline__ float d2f_rn(double d) {
  const uint64_t u = bits_of(d);
  const uint32_t s = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FFu);
  const uint64_t m = u & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return float_of(s | 0x7F800000u | (m ? 0x400000u : 0u));
  const int E = e - 1023;
  if (E > 127) return float_of(s | 0x7F800000u);
  if (E >= -126) {
    // normal result: keep 23 of the 52 fraction bits; a carry out of the fraction
    // raises the exponent (at the top of the range it gives infinity)
    const uint32_t q = (uint32_t)(m >> 29), r = (uint32_t)(m & 0x1FFFFFFFu);
    uint32_t v = ((uint32_t)(E + 127) << 23) | q;
    if (r > 0x10000000u || (r == 0x10000000u && (q & 1u))) ++v;
    return float_of(s | v);
  }
  if (E < -150) return float_of(s);  // below half the smallest subnormal
  // subnormal result: the significand (2^52 + m) in units of 2^-149 is shifted right
  // by sh = -E - 97 (30 .. 53) and rounded; rounding up from the largest subnormal
  // gives the smallest normal number, whose bits follow on
  const uint64_t M = (1ull << 52) | m;
  const int sh = -E - 97;
  uint32_t q = (uint32_t)(M >> sh);
  const uint64_t r = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  if (r > half || (r == half && (q & 1u))) ++q;
  return float_of(s | q);
}

}  // namespace pbs
