// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.  Built on the
// error-free transformations of Knuth (two-sum) and Dekker (two-product, here
// with a fused multiply-add); sums use the cheap form whose relative error stays
// near 2^-44 of the larger operand.  Used where GB300's FP64 rate is too low for
// per-tile work that needs more than FP32: every operation runs on the FP32 pipes.
// Requires IEEE FP32 without reassociation (no fast-math); fused multiply-adds are
// written out explicitly.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace ecc {

struct df {
  float hi, lo;
};

__host__ __device__ __forceinline__ float df_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

__host__ __device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

__host__ __device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return {s, b - (s - a)};
}

__host__ __device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = a * b;
  return {p, df_fma(a, b, -p)};
}

__host__ __device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return df_fast_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

__host__ __device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__host__ __device__ __forceinline__ df df_mul(df a, df b) {
  df p = df_two_prod(a.hi, b.hi);
  p.lo = df_fma(a.hi, b.lo, p.lo);
  p.lo = df_fma(a.lo, b.hi, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}

__host__ __device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = df_two_prod(a.hi, b);
  p.lo = df_fma(a.lo, b, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}

// Split of an FP64 value (exact to about 2^-48 relative).
__host__ __device__ __forceinline__ df df_from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

__host__ __device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// 1 / a from an FP32 reciprocal and one Newton step in double-float.
__host__ __device__ __forceinline__ df df_recip(df a) {
  const float r0 = 1.0f / a.hi;
  const df e = df_sub(df{1.0f, 0.0f}, df_mul_f(a, r0));  // 1 - a r0, small
  return df_add(df{r0, 0.0f}, df_mul_f(e, r0));
}

// 1 / sqrt(a), a > 0, from an FP32 estimate and one Newton step in double-float.
__host__ __device__ __forceinline__ df df_rsqrt(df a) {
#ifdef __CUDA_ARCH__
  const float y0 = rsqrtf(a.hi);
#else
  const float y0 = 1.0f / std::sqrt(a.hi);
#endif
  const df ay2 = df_mul_f(df_mul_f(a, y0), y0);                    // a y0^2, close to 1
  const df t = df_sub(df{1.5f, 0.0f}, df_mul_f(ay2, 0.5f));        // 3/2 - a y0^2 / 2
  return df_mul_f(t, y0);
}

// floor of a double-float value and the FP32 fraction in [0, 1).
__host__ __device__ __forceinline__ float df_floor_frac(df a, float* frac) {
  float n = floorf(a.hi);
  float f = (a.hi - n) + a.lo;  // a.hi - n is exact below 2^23
  if (f < 0.0f) {
    n -= 1.0f;
    f += 1.0f;
  } else if (f >= 1.0f) {
    n += 1.0f;
    f -= 1.0f;
  }
  *frac = f;
  return n;
}

}  // namespace ecc
