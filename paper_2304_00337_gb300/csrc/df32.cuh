// Double-float ("df32") arithmetic: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits (relative
// rounding ~ 3.6e-15).  On GB300 an FP64 warp instruction occupies the FP64
// pipe for ~64 cycles while an FP32 one issues every cycle, so kernels whose
// accuracy needs are below 1e-14 (Gram matrices, the small Rayleigh-Ritz
// eigensolve, the projection right-hand side) run on the FP32 pipe with these
// operations.  Built from the standard error-free transformations: Knuth's
// two-sum (exact a + b = s + e) and the FMA two-product (exact a * b = p + e).
#pragma once
#include "fpconv.cuh"
#include <cuda_runtime.h>

namespace pbs {

struct df {
  float hi, lo;
  df() = default;
  // rounding of a double to hi + lo; meant for constants (folded at compile time)
  __host__ __device__ constexpr explicit df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

__device__ __forceinline__ df df_make(float h, float l) {
  df r;
  r.hi = h;
  r.lo = l;
  return r;
}
__device__ __forceinline__ df df_from(double d) {
  const float h = (float)d;
  return df_make(h, (float)(d - (double)h));
}
// hi + lo in FP64; the widening of the two floats is exact and done by integer
// operations (fpconv.cuh), so only the sum uses the FP64 pipe
__device__ __forceinline__ double df_to(df a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }

// exact s + e = a + b (no ordering requirement)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
// exact s + e = a + b when |a| >= |b| or a == 0
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// exact p + e = a * b
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df_make(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ df operator+(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df operator-(df a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
// a / b: one float quotient corrected twice against the df remainder
__device__ __forceinline__ df operator/(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  df r = a - df_mul_f(b, q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  r = r - df_mul_f(b, q2);
  const float q3 = __fdiv_rn(r.hi, b.hi);
  df q = quick_two_sum(q1, q2);
  return q + df_make(q3, 0.0f);
}
// sqrt(a), a >= 0: float estimate plus one Newton correction in df
__device__ __forceinline__ df df_sqrt(df a) {
  if (a.hi <= 0.0f) return df_make(0.0f, 0.0f);
  const float x = __fsqrt_rn(a.hi);
  const df x2 = two_prod(x, x);
  const df r = a - x2;
  const float c = __fdiv_rn(r.hi, 2.0f * x);
  return quick_two_sum(x, c);
}
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ df df_abs(df a) { return a.hi < 0.0f ? -a : a; }
__device__ __forceinline__ df df_zero() { return df_make(0.0f, 0.0f); }

// FP64 -> df with integer operations only (no FP64 instruction): hi keeps the
// leading 24 significand bits of d (truncated), lo the next 24 rounded to nearest,
// so |d - (hi + lo)| <= 2^-47 |d|.  Magnitudes below 2^-100 give 0; magnitudes in
// [2^127, 2^128) give their leading 24 bits alone, larger ones infinity (NaN stays
// NaN) - all without an FP64 instruction.
__device__ __forceinline__ df df_split(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
  const int e = (int)((hw >> 20) & 0x7FFu) - 1023;
  if (e < -100) return df_make(0.0f, 0.0f);
  const unsigned sgn = hw & 0x80000000u;
  if (__builtin_expect(e > 126, 0)) {
    // |d| >= 2^127: the leading 24 bits alone; beyond the binary32 range infinity
    // (NaN stays NaN).  A few integer operations, cheap where the compiler predicates them.
    const unsigned over = sgn | 0x7F800000u | ((e == 1024 && ((hw & 0xFFFFFu) | lw)) ? 0x400000u : 0u);
    const unsigned top = sgn | (254u << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    return df_make(__uint_as_float(e > 127 ? over : top), 0.0f);
  }
  const float hi = __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  // the remaining 29 bits r scaled by 2^(e-52): round to 23 bits and place them under
  // the implicit bit of 2^(e-23); a carry out of the 23 bits moves into the exponent,
  // which is still the right value.  The subtraction is exact (Sterbenz).
  const unsigned base = sgn | ((unsigned)(e + 104) << 23);
  const unsigned r = lw & 0x1FFFFFFFu;
  const float lo = __fsub_rn(__uint_as_float(base + ((r + 32u) >> 6)), __uint_as_float(base));
  return quick_two_sum(hi, lo);
}

// Streaming arithmetic: a + b with one two-sum on the leading parts and a plain
// float sum of the trailing parts; its error is about 2^-47 (|a| + |b|), which is
// the measure every stencil and block kernel needs (errors relative to the
// vectors' norms, not to a cancelled result).
__device__ __forceinline__ df dfs_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df dfs_sub(df a, df b) { return dfs_add(a, df_make(-b.hi, -b.lo)); }
__device__ __forceinline__ float df_to_float(df a) { return __fadd_rn(a.hi, a.lo); }

// Complex value of the streaming kernels (members x = re, y = im, like float2 /
// double2, so the templated stencils instantiate with it).
struct dcx {
  df x, y;
};
__device__ __forceinline__ dcx dcx_make(df r, df i) {
  dcx z;
  z.x = r;
  z.y = i;
  return z;
}
__device__ __forceinline__ dcx operator+(dcx a, dcx b) { return dcx_make(dfs_add(a.x, b.x), dfs_add(a.y, b.y)); }
__device__ __forceinline__ dcx operator-(dcx a, dcx b) { return dcx_make(dfs_sub(a.x, b.x), dfs_sub(a.y, b.y)); }
__device__ __forceinline__ dcx operator-(dcx a) { return dcx_make(-a.x, -a.y); }
__device__ __forceinline__ dcx operator*(df s, dcx a) { return dcx_make(s * a.x, s * a.y); }
__device__ __forceinline__ dcx cmul(dcx a, dcx b) {
  return dcx_make(dfs_sub(a.x * b.x, a.y * b.y), dfs_add(a.x * b.y, a.y * b.x));
}
__device__ __forceinline__ dcx conj(dcx a) { return dcx_make(a.x, -a.y); }
__device__ __forceinline__ df nrm2(dcx a) { return dfs_add(a.x * a.x, a.y * a.y); }
__device__ __forceinline__ dcx dcx_split(double2 v) { return dcx_make(df_split(v.x), df_split(v.y)); }
__device__ __forceinline__ double2 dcx_to(dcx v) { return make_double2(df_to(v.x), df_to(v.y)); }

// Compensated dot-product accumulator (the Dot2 scheme of Ogita, Rump and Oishi,
// 2005, with df operands): s collects the leading products by two-sums, c the
// rounding errors of those sums and products and the cross terms with the
// trailing parts.  s + c carries about twice the float precision as long as c is
// folded back (dot2_fold) every few dozen terms.
struct acc2 {
  float s, c;
};
__device__ __forceinline__ acc2 acc2_zero() {
  acc2 a;
  a.s = 0.0f;
  a.c = 0.0f;
  return a;
}
// a += x * y
__device__ __forceinline__ void dot2(acc2& a, df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float pe = __fmaf_rn(x.hi, y.hi, -p);
  const float t = __fadd_rn(a.s, p);
  const float z = __fsub_rn(t, a.s);
  const float se = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(p, z));
  a.s = t;
  a.c = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, __fadd_rn(a.c, __fadd_rn(pe, se))));
}
// a -= x * y
__device__ __forceinline__ void dot2_neg(acc2& a, df x, df y) { dot2(a, df_make(-x.hi, -x.lo), y); }
__device__ __forceinline__ void dot2_fold(acc2& a) {
  const df r = two_sum(a.s, a.c);
  a.s = r.hi;
  a.c = r.lo;
}
__device__ __forceinline__ df acc2_df(acc2 a) { return two_sum(a.s, a.c); }

// complex double-float
struct cdf {
  df re, im;
};
__device__ __forceinline__ cdf cdf_make(df r, df i) {
  cdf z;
  z.re = r;
  z.im = i;
  return z;
}
__device__ __forceinline__ cdf cdf_from(double2 v) { return cdf_make(df_from(v.x), df_from(v.y)); }
__device__ __forceinline__ double2 cdf_to(cdf z) { return make_double2(df_to(z.re), df_to(z.im)); }
__device__ __forceinline__ cdf cdf_zero() { return cdf_make(df_zero(), df_zero()); }
__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return cdf_make(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return cdf_make(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cdf operator-(cdf a) { return cdf_make(-a.re, -a.im); }
__device__ __forceinline__ cdf cdf_conj(cdf a) { return cdf_make(a.re, -a.im); }
__device__ __forceinline__ cdf operator*(cdf a, cdf b) {
  return cdf_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// conj(a) * b
__device__ __forceinline__ cdf cdf_mulc(cdf a, cdf b) {
  return cdf_make(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
__device__ __forceinline__ cdf cdf_scale(cdf a, df s) { return cdf_make(a.re * s, a.im * s); }
__device__ __forceinline__ df cdf_norm2(cdf a) { return a.re * a.re + a.im * a.im; }

}  // namespace pbs
