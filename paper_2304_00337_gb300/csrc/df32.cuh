// Double-float ("df32") arithmetic: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, about 48 significant bits (relative
// rounding ~ 3.6e-15).  On GB300 an FP64 warp instruction occupies the FP64
// pipe for ~64 cycles while an FP32 one issues every cycle, so kernels whose
// accuracy needs are below 1e-14 (Gram matrices, the small Rayleigh-Ritz
// eigensolve, the projection right-hand side) run on the FP32 pipe with these
// operations.  Built from the standard error-free transformations: Knuth's
// two-sum (exact a + b = s + e) and the FMA two-product (exact a * b = p + e).
#pragma once
#include <cuda_runtime.h>

namespace pbs {

struct df {
  float hi, lo;
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
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }

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
