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

// a / b for an FP32 divisor (one correction of the FP32 quotient).
__host__ __device__ __forceinline__ df df_div_f(df a, float b) {
  const float q1 = a.hi / b;
  const df p = df_two_prod(q1, b);
  const float r = ((a.hi - p.hi) - p.lo) + a.lo;
  return df_fast_two_sum(q1, r / b);
}

__host__ __device__ __forceinline__ bool df_lt0(df a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f); }

// pi as a double-float pair; pi / 2 in three FP32 parts (for the range reduction);
// all folded at compile time (scalar constexpr values).
constexpr double kDfPi = 3.14159265358979323846;
constexpr float kDfPiHi = (float)kDfPi;
constexpr float kDfPiLo = (float)(kDfPi - (double)kDfPiHi);
constexpr double kDfPio2 = 1.57079632679489661923;
constexpr float kDfPio2A = (float)kDfPio2;
constexpr float kDfPio2B = (float)(kDfPio2 - (double)kDfPio2A);
constexpr float kDfPio2C = (float)((kDfPio2 - (double)kDfPio2A) - (double)kDfPio2B);
constexpr float kDf2OverPi = (float)(2.0 / kDfPi);

__host__ __device__ inline df df_pi() { return df{kDfPiHi, kDfPiLo}; }

// 1 / n! at compile time.
template <int N>
struct DfInvFact {
  static constexpr double v = DfInvFact<N - 1>::v / (double)N;
};
template <>
struct DfInvFact<0> {
  static constexpr double v = 1.0;
};

// Horner forms of sum_{j >= k} (-1)^j x^j / (2j + 1)! (sin r / r, x = r^2, to j = 8)
// and of sum_{j >= k} (-1)^j x^j / (2j)! (cos r, to j = 9), coefficients as
// double-float constants.
template <int k>
__host__ __device__ __forceinline__ df df_sin_poly(df x) {
  constexpr double c = ((k & 1) ? -1.0 : 1.0) * DfInvFact<2 * k + 1>::v;
  constexpr float ch = (float)c, cl = (float)(c - (double)ch);
  if constexpr (k == 8)
    return df{ch, cl};
  else
    return df_add(df_mul(df_sin_poly<k + 1>(x), x), df{ch, cl});
}
template <int k>
__host__ __device__ __forceinline__ df df_cos_poly(df x) {
  constexpr double c = ((k & 1) ? -1.0 : 1.0) * DfInvFact<2 * k>::v;
  constexpr float ch = (float)c, cl = (float)(c - (double)ch);
  if constexpr (k == 9)
    return df{ch, cl};
  else
    return df_add(df_mul(df_cos_poly<k + 1>(x), x), df{ch, cl});
}

// sin and cos of a double-float angle |a| <= 4: a = q pi/2 + r with |r| <= pi/4 (q an
// integer, r in double-float), Taylor series of sin r to r^17 and of cos r to r^18
// (truncation below 1e-16 at |r| = pi/4), then the quadrant.  Not inlined: one copy of
// the series serves every call (a kernel that inlined five copies waited on
// instruction fetch).
__host__ __device__ inline __noinline__ void df_sincos(df a, df* s, df* c) {
  const float q = rintf(a.hi * kDf2OverPi);
  const df qp = df_add(df_add(df_two_prod(q, kDfPio2A), df_two_prod(q, kDfPio2B)), df{q * kDfPio2C, 0.0f});
  const df r = df_sub(a, qp);
  const df x = df_mul(r, r);
  const df sr = df_mul(df_sin_poly<0>(x), r), cr = df_cos_poly<0>(x);
  const int qi = ((int)q) & 3;
  *s = qi == 0 ? sr : (qi == 1 ? cr : (qi == 2 ? df_neg(sr) : df_neg(cr)));
  *c = qi == 0 ? cr : (qi == 1 ? df_neg(sr) : (qi == 2 ? df_neg(cr) : sr));
}

// atan2(y, x) in double-float: the FP32 angle t0 and its sin and cos, then the
// remaining turn d = atan((y cos t0 - x sin t0) / (x cos t0 + y sin t0)); |d| is a few
// 1e-7, so d itself (error d^3 / 3) completes it.  atan2(0, 0) = 0.
__host__ __device__ inline __noinline__ df df_atan2(df y, df x) {
  if (y.hi == 0.0f && x.hi == 0.0f) return df{0.0f, 0.0f};
  const float t0 = atan2f(y.hi, x.hi);
  df s0, c0;
  df_sincos(df{t0, 0.0f}, &s0, &c0);
  const df num = df_sub(df_mul(y, c0), df_mul(x, s0));
  const df den = df_add(df_mul(x, c0), df_mul(y, s0));
  return df_add(df{t0, 0.0f}, df_mul(num, df_recip(den)));
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
