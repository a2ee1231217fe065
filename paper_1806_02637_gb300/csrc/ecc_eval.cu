// Pair x kappa gather-reduce of the epipolar consistency metric (Eq. 15-17).
//
// The pair's K sampled planes are processed in tiles: of 64 planes in the forward
// kernel (two per lane; a warp owns one or two pairs), of 32 in the adjoint (one per
// lane; a warp owns one pair).  For every tile and view the line of the tile centre is
// a double-float "anchor" (computed lane-parallel, one anchor per lane), split into
// an exact (alpha row, s bin) integer part and an FP32 fraction, with the series of
// the tile's offsets in t = tan(delta); each lane then moves from the anchor to its
// own plane in FP32, so that the sinogram indices carry FP64-class accuracy while
// the per-sample work stays in FP32.  Bilinear taps are gathered from the
// sinograms, squared differences are accumulated in FP32, reduced with warp
// shuffles, normalised by N_kappa (Eq. 15), passed through the Cauchy norm (Eq. 16)
// and summed per block in a fixed order (Eq. 17, finished by the reduce kernel).
// The adjoint variant also accumulates d e / d A for the gradient kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ecc_internal.cuh"
#include "df.cuh"
#include "kernels.cuh"

namespace ecc {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kPairsPerForwardBlock = 2 * kWarpsPerBlock;  // the forward kernel: two pairs per warp
constexpr int kForwardWavesForTwo = 3;  // ... when that leaves at least this many waves of blocks
// 64-sample tiles reach 31.5 dk from their anchor, dk <= pi / n_kappa; the closed form
// needs |delta| < pi / 2.  From 96 samples on that is at most 1.03 rad; smaller n_kappa
// take the adjoint's 32-sample tiles (15.5 dk), without its gradient output.
constexpr int kMinKappaForward64 = 96;

template <typename T>
struct Elem;
template <>
struct Elem<float> {
  static __device__ __forceinline__ float get(const float* p) { return __ldg(p); }
};
template <>
struct Elem<__half> {
  static __device__ __forceinline__ float get(const __half* p) { return __half2float(__ldg(p)); }
};
template <>
struct Elem<__nv_bfloat16> {
  static __device__ __forceinline__ float get(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
};

// Bilinear value at alpha row m (+ fraction fa toward row m+1) and s position
// n + fs of one view's sinogram.  Row n_alpha continues as row 0 at -s, negated.
// A line that meets the detector lies inside the s grid (|s| <= half its diagonal),
// so the bin is clamped to [0, n_s - 2] once instead of testing every tap: this
// changes nothing for such lines and keeps the reads of masked samples in bounds.
template <typename T>
__device__ __forceinline__ float bilinear(const T* __restrict__ sv, int n_alpha, int n_s, int m, float fa, int n,
                                          float fs) {
  n = min(max(n, 0), n_s - 2);
  const T* r0 = sv + (size_t)m * n_s + n;
  const float t00 = Elem<T>::get(r0), t01 = Elem<T>::get(r0 + 1);
  const float v0 = fmaf(fs, t01 - t00, t00);
  float v1;
  if (m + 1 < n_alpha) {
    const float t10 = Elem<T>::get(r0 + n_s), t11 = Elem<T>::get(r0 + n_s + 1);
    v1 = fmaf(fs, t11 - t10, t10);
  } else {  // row 0 at bins n_s - 1 - n and n_s - 2 - n
    const T* q = sv + (n_s - 2 - n);
    const float t10 = Elem<T>::get(q + 1), t11 = Elem<T>::get(q);
    v1 = -fmaf(fs, t11 - t10, t10);
  }
  return fmaf(fa, v1 - v0, v0);
}

constexpr int kSer = 16;  // terms of the per-tile series (at most)
// The series is used while rho = |zeta| tan(half tile) is at most this (else the closed
// form per sample): 0.2 for the forward's 64-sample tiles (up to 16 terms: the tail
// after them stays below 1e-8 bins), 0.1 for the adjoint's 32-sample tiles (up to 10
// terms), whose rho is half as large.
constexpr float kSerLimit64 = 0.2f;
constexpr float kSerLimit32 = 0.1f;
// The s index advances by gh jj + gl jj per sample offset jj; gh keeps few enough
// significant bits that gh jj is exact in FP32: 18 for the adjoint's 32-sample tiles
// (2 jj an integer below 2^5), 16 for the forward's 64-sample tiles (4 jj an integer
// below 2^8).
constexpr unsigned kGhMask32 = 0xffffffc0u;
constexpr unsigned kGhMask64 = 0xffffff00u;

// Per (tile, view) anchor record, 44 floats (176 B), written by one lane and read by
// the whole warp through shared memory.  The fields of the series path come first.
struct Anchor {
  int m0, n0;      // alpha row and s bin of the tile-centre line
  float fa0, fs0;  // fractional parts (may leave [0,1) slightly)
  float sg;        // orientation fold of the anchor (+1 / -1)
  float gh, gl;    // exact s-index advance per sample step: gh (17 significant bits) + gl
  float ser;       // number of series terms that hold over this tile (2 .. kSer), 0: closed form per sample
  float dco[kSer];  // alpha offset [bins] = sum_k dco[k-1] t^k,  t = tan(delta); zero beyond ser terms
  float sco[kSer];  // s remainder [bins] = sco[0] (t - delta) + sum_{k>=2} sco[k-1] t^k; zero beyond ser
  float a, b;      // zeta = a + i b: rate of the normal direction in the anchor frame
  float p3, s0;    // rate of the offset, anchor offset s [px]
};
static_assert(sizeof(Anchor) == 176, "anchor record is 44 floats");
constexpr int kRec = sizeof(Anchor) / sizeof(float4);  // float4 words per record

union AnchorVec {
  Anchor a;
  float4 v[kRec];
};

__device__ __forceinline__ void store_anchor(float4* __restrict__ dst, const Anchor& x) {
  AnchorVec u;
  u.a = x;
#pragma unroll
  for (int i = 0; i < kRec; ++i) dst[i] = u.v[i];
}

__device__ __forceinline__ Anchor load_anchor(const float4* __restrict__ src) {
  AnchorVec u;
#pragma unroll
  for (int i = 0; i < kRec; ++i) u.v[i] = src[i];
  return u.a;
}

// Anchor of one (view, tile): the epipolar line l = A c (centred detector
// coordinates) of the tile-centre plane, folded to alpha in [0, pi), located on the
// alpha grid against the exact row direction, and its s offset.  The construction
// needs more than FP32 (l is a sum of products of FP64-sized terms, and the s index
// must hold 1e-7 bins over hundreds of bins), and GB300 issues FP64 at 1/64 of the
// FP32 rate, so it runs in double-float arithmetic (about 48 bits) on the FP32
// pipes; A, c and the row directions arrive split into (hi, lo) pairs.
__device__ Anchor make_anchor(const float* __restrict__ Adf, float4 c, const float4* __restrict__ alpha_dir,
                              int n_alpha, float inv_dalpha, df inv_ds, df half_ns1, float inv_ds_f, df dk,
                              float tan_half_tile, unsigned gh_mask, float ser_limit, int max_terms) {
  const df cx = {c.x, c.z}, cy = {c.y, c.w};
  const df A0 = {Adf[0], Adf[1]}, A1 = {Adf[2], Adf[3]}, A2 = {Adf[4], Adf[5]};
  const df A3 = {Adf[6], Adf[7]}, A4 = {Adf[8], Adf[9]}, A5 = {Adf[10], Adf[11]};
  df l0 = df_add(df_mul(A0, cx), df_mul(A1, cy));
  df l1 = df_add(df_mul(A2, cx), df_mul(A3, cy));
  df l2 = df_add(df_mul(A4, cx), df_mul(A5, cy));
  // derivative of the line with respect to kappa: A c_perp, c_perp = (-c.y, c.x)
  df p0 = df_sub(df_mul(A1, cx), df_mul(A0, cy));
  df p1 = df_sub(df_mul(A3, cx), df_mul(A2, cy));
  df p2 = df_sub(df_mul(A5, cx), df_mul(A4, cy));
  Anchor r;
  r.sg = 1.0f;
  if (l1.hi < 0.0f || (l1.hi == 0.0f && l0.hi < 0.0f)) {
    l0 = df_neg(l0); l1 = df_neg(l1); l2 = df_neg(l2);
    p0 = df_neg(p0); p1 = df_neg(p1); p2 = df_neg(p2);
    r.sg = -1.0f;
  }
  const float l0f = l0.hi, l1f = l1.hi;
  const float q0 = p0.hi, q1 = p1.hi, q2 = p2.hi;
  const float h = sqrtf(l0f * l0f + l1f * l1f);
  const float ih_f = 1.0f / h;
  const float chx = l0f * ih_f, chy = l1f * ih_f;
  r.a = (q0 * chx + q1 * chy) * ih_f;
  r.b = (q1 * chx - q0 * chy) * ih_f;
  r.p3 = q2 * ih_f;
  int m = (int)floorf(atan2f(l1f, l0f) * inv_dalpha);
  m = m < 0 ? 0 : (m > n_alpha - 1 ? n_alpha - 1 : m);
  const float4 u = alpha_dir[m];
  const df ux = {u.x, u.z}, uy = {u.y, u.w};
  const df cr = df_sub(df_mul(ux, l1), df_mul(uy, l0));  // h sin(alpha - alpha_m)
  const df dt = df_add(df_mul(ux, l0), df_mul(uy, l1));  // h cos(alpha - alpha_m)
  // turn th from the row direction: within about one alpha bin, so atan, sin(th/2)
  // and cos(th) = 1 - 2 sin^2(th/2) come from short odd/even series (truncation below
  // 1e-12 relative for |th| <= 0.05); wider turns (coarse alpha grids) use the library
  const float xr = cr.hi / dt.hi;
  float th, sh;
  if (fabsf(xr) <= 0.05f && dt.hi > 0.0f) {
    const float x2 = xr * xr;
    th = xr * fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 7.0f, 1.0f / 5.0f), -1.0f / 3.0f), 1.0f);
    const float y = 0.5f * th, y2 = y * y;
    sh = y * fmaf(y2, fmaf(y2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
  } else {
    th = atan2f(cr.hi, dt.hi);
    sh = sinf(0.5f * th);
  }
  r.m0 = m;
  r.fa0 = th * inv_dalpha;
  // s = -l2 / h = (-l2 / dt) cos(th)
  const df sigma = df_neg(df_mul(l2, df_recip(dt)));
  float frac;
  const float nf = df_floor_frac(df_add(df_mul(sigma, inv_ds), half_ns1), &frac);
  const float sigf = sigma.hi;
  const float vers = 2.0f * sh * sh;  // 1 - cos(th)
  r.n0 = (int)fminf(fmaxf(nf, -4.0e6f), 4.0e6f);  // a masked tile centre may lie far outside
  r.fs0 = frac - sigf * vers * inv_ds_f;
  r.s0 = sigf * (1.0f - vers);
  // exact first-order advance of the s index per sample: (ds/dkappa) dk / ds_bin,
  // ds/dkappa = (1/h) (-l2' + l2 (l . l') / h^2)
  const df ih = df_rsqrt(df_add(df_mul(l0, l0), df_mul(l1, l1)));
  const df t1 = df_add(df_mul(l0, p0), df_mul(l1, p1));
  const df g = df_mul(df_mul(df_mul(ih, df_sub(df_mul(df_mul(l2, t1), df_mul(ih, ih)), p2)), dk), inv_ds);
  const float gh = __int_as_float((int)((unsigned)__float_as_int(g.hi) & gh_mask));
  r.gh = gh;
  r.gl = (g.hi - gh) + g.lo;
  // Series over the tile in t = tan(delta).  In the anchor frame the normal of the
  // line at delta is cos(delta) (1 + zeta t), zeta = a + i b, so the alpha offset is
  // arg(1 + zeta t) = sum_k (-1)^(k+1) Im(zeta^k) t^k / k, and
  //   s(t) = (s0 - p3 t) / |1 + zeta t| = (s0 - p3 t) sum_k e_k t^k,
  // where (1 + 2 a t + |zeta|^2 t^2)^(-1/2) = sum_k e_k t^k is the Legendre generating
  // function: e_0 = 1, e_1 = -a, (k + 1) e_(k+1) = -((2k + 1) a e_k + k |zeta|^2 e_(k-1)).
  // With |zeta t| <= 0.2 the truncation after t^16 is below 1e-11 of the offsets.
  const float zr = r.a, zi = r.b;
  const float z2 = fmaf(zr, zr, zi * zi);
  // Terms needed: with rho = |zeta| tan(half tile) the k-th terms are bounded by
  // rho^k inv_dalpha (alpha) and (|s0| rho^k + |p3| t rho^(k-1)) inv_ds (s), since
  // |Im zeta^k| <= |zeta|^k and |e_k| <= |zeta|^k; the tails after n terms are these
  // geometric sums.  The smallest n >= 2 whose tail bound is below 1e-8 bins is kept,
  // at most max_terms (the s index carries ~6e-8 bins of FP32 rounding anyway).
  const float rho = sqrtf(z2) * tan_half_tile;
  int nser = 0;
  if (tan_half_tile >= 0.0f && rho <= ser_limit && isfinite(r.s0) && isfinite(r.fs0) && isfinite(r.fa0)) {
    const float cs = fabsf(r.s0) * inv_ds_f, cp = fabsf(r.p3) * tan_half_tile * inv_ds_f;
    const float inv1m = 1.0f / (1.0f - rho);
    float rn = rho * rho;  // rho^n for n = 2
    nser = 2;
    while (nser < max_terms && ((inv_dalpha + cs) * rn * rho + cp * rn) * inv1m > 1e-8f) {
      rn *= rho;
      ++nser;
    }
  }
  r.ser = (float)nser;
#pragma unroll
  for (int k = 0; k < kSer; ++k) r.dco[k] = r.sco[k] = 0.0f;
  float pre = zr, pim = zi;        // zeta^k
  float e_prev = 1.0f, e_cur = -zr;  // e_(k-1), e_k
#pragma unroll
  for (int k = 1; k <= kSer; ++k) {
    if (k > nser) break;
    r.dco[k - 1] = ((k & 1) ? pim : -pim) * inv_dalpha * (1.0f / (float)k);
    r.sco[k - 1] = fmaf(r.s0, e_cur, -r.p3 * e_prev) * inv_ds_f;
    const float e_next = -fmaf((float)(2 * k + 1) * zr, e_cur, (float)k * z2 * e_prev) * (1.0f / (float)(k + 1));
    e_prev = e_cur;
    e_cur = e_next;
    const float np = fmaf(pre, zr, -pim * zi), ni = fmaf(pre, zi, pim * zr);
    pre = np;
    pim = ni;
  }
  return r;
}

// Position of one sample of one view in the sinogram grid, moving from the tile
// anchor by delta = jj dk (jj a half-integer lane offset).  The s index splits into
// the exact first-order part jj * (gh + gl) (gh * jj is exact in FP32, its integer
// part split off exactly) and a remainder of second order in delta; the alpha
// index is the anchor's plus the turn of the normal.  Two evaluations:
//   series (locate_series): both from the anchor's series in t = tan(delta);
//   closed form (locate): the turn atan2(b sd, cd + a sd) and the remainder in a
//   cancellation-free form,
//     ds - G1 delta = -(s0 q + p3) u - s0 (q - a) delta,
//     u = sd/r - delta = ((sin delta - delta) - delta (r - 1)) / r,
//     r^2 - 1 = sd (2 a cd + (a^2 + b^2 - 1) sd),  q = (2 a cd + (a^2 + b^2) sd)/(cd + r).
struct Loc {
  int m, n;
  float fa, fs, sign;
  bool ok;
};

// Row/bin split of the fractional indices and the fold of alpha into [0, pi).
__device__ __forceinline__ Loc loc_tail(const Anchor& an, float fa, float fs, float Li, int n_alpha, int n_s) {
  // masked samples of the other view may carry extreme offsets: clamp before the
  // integer conversion so that no index arithmetic can overflow
  const float mfl = fminf(fmaxf(floorf(fa), -4.0e6f), 4.0e6f);
  const float nfl = fminf(fmaxf(floorf(fs), -4.0e6f), 4.0e6f);
  const float lif = fminf(fmaxf(Li, -4.0e6f), 4.0e6f);
  Loc o;
  o.m = an.m0 + (int)mfl;
  o.n = an.n0 + (int)lif + (int)nfl;
  o.fa = fa - mfl;
  o.fs = fs - nfl;
  o.sign = an.sg;
  if (o.m >= n_alpha || o.m < 0) {  // alpha left [0, pi): S(alpha + pi, s) = -S(alpha, -s)
    o.m += o.m < 0 ? n_alpha : -n_alpha;
    o.n = n_s - 2 - o.n;
    o.fs = 1.0f - o.fs;
    o.sign = -o.sign;
  }
  o.ok = o.m >= 0 && o.m < n_alpha;  // false only for a masked sample
  return o;
}

__device__ __forceinline__ Loc locate(const Anchor& an, float cd, float sd, float jj, float de, int n_alpha,
                                      int n_s, float inv_dalpha, float inv_ds_f) {
  const float x = fmaf(an.a, sd, cd);
  const float y = an.b * sd;
  const float dal = atan2f(y, x);
  const float ab2 = fmaf(an.a, an.a, an.b * an.b);
  const float r2m1 = sd * fmaf(2.0f * an.a, cd, (ab2 - 1.0f) * sd);
  const float r = sqrtf(1.0f + r2m1);
  const float rm1 = __fdividef(r2m1, r + 1.0f);
  const float cpr = cd + r;
  const float q = __fdividef(fmaf(2.0f * an.a, cd, ab2 * sd), cpr);
  const float qma = sd * __fdividef(fmaf(-an.a, q, ab2), cpr);
  const float d2 = de * de;
  // sin(delta) - delta by its Taylor series to delta^13 (relative truncation below
  // 4e-8 for |delta| <= 1.5, the widest tile of a full-pi arc with K >= 32)
  float sdmd = fmaf(d2, 1.0f / 6227020800.0f, -1.0f / 39916800.0f);
  sdmd = fmaf(d2, sdmd, 1.0f / 362880.0f);
  sdmd = fmaf(d2, sdmd, -1.0f / 5040.0f);
  sdmd = fmaf(d2, sdmd, 1.0f / 120.0f);
  sdmd = fmaf(d2, sdmd, -1.0f / 6.0f);
  sdmd *= de * d2;
  const float u = __fdividef(fmaf(-de, rm1, sdmd), r);
  const float R = -fmaf(an.s0, q, an.p3) * u - an.s0 * qma * de;
  const float lin = an.gh * jj;  // exact
  const float Li = floorf(lin);
  const float Lf = lin - Li;     // exact
  const float fa = fmaf(dal, inv_dalpha, an.fa0);
  const float fs = (an.fs0 + Lf) + fmaf(an.gl, jj, R * inv_ds_f);
  return loc_tail(an, fa, fs, Li, n_alpha, n_s);
}

// t = tan(delta), tmd = tan(delta) - delta (accurate for small delta).
__device__ __forceinline__ Loc locate_series(const Anchor& an, float t, float tmd, float jj, int n_alpha, int n_s) {
  float da = an.dco[kSer - 1];
#pragma unroll
  for (int k = kSer - 2; k >= 0; --k) da = fmaf(da, t, an.dco[k]);
  da *= t;
  float sr = an.sco[kSer - 1];
#pragma unroll
  for (int k = kSer - 2; k >= 1; --k) sr = fmaf(sr, t, an.sco[k]);
  sr = fmaf(an.sco[0], tmd, (t * t) * sr);
  const float lin = an.gh * jj;  // exact
  const float Li = floorf(lin);
  const float Lf = lin - Li;     // exact
  const float fa = an.fa0 + da;
  const float fs = (an.fs0 + Lf) + fmaf(an.gl, jj, sr);
  return loc_tail(an, fa, fs, Li, n_alpha, n_s);
}

// tan(delta) - delta: Taylor series below 0.25 (no cancellation), else direct.
__device__ __forceinline__ float tan_minus_angle(float d, float t) {
  const float d2 = d * d;
  float p = fmaf(d2, 1382.0f / 155925.0f, 62.0f / 2835.0f);
  p = fmaf(d2, p, 17.0f / 315.0f);
  p = fmaf(d2, p, 2.0f / 15.0f);
  p = fmaf(d2, p, 1.0f / 3.0f);
  return fabsf(d) < 0.25f ? d * d2 * p : t - d;
}

// One sample of one view: locate it and gather the bilinear value.
template <typename T>
__device__ __forceinline__ float sample(const T* __restrict__ sv, int n_alpha, int n_s, const Loc& o) {
  if (!o.ok) return 0.0f;
  return o.sign * bilinear(sv, n_alpha, n_s, o.m, o.fa, o.n, o.fs);
}

// Value and gradient of one sample with respect to its line l = A c (centred
// detector coordinates) for the adjoint.  The look-up is evaluated at the folded
// line L = sigma l (sigma = product of the orientation folds, the same sign that
// multiplies the value), so dS/dl = B_alpha d(alpha)/dL + B_s d(s)/dL at L with
// d(alpha)/dL = (-sin a, cos a, 0)/h and d(s)/dL = -(s cos a, s sin a, 1)/h;
// B_alpha, B_s are the slopes of the bilinear cell (piecewise constant).
template <typename T>
__device__ __forceinline__ float sample_grad(const T* __restrict__ sv, int n_alpha, int n_s, const Loc& o,
                                             float inv_dalpha, float inv_ds_f, float l0, float l1, float l2,
                                             float scale, float* g) {
  const int m = o.m;
  const int n = min(max(o.n, 0), n_s - 2);  // as in bilinear()
  const float fa = o.fa, fs = o.fs, sign = o.sign;
  g[0] = g[1] = g[2] = 0.0f;
  if (!o.ok) return 0.0f;
  const T* r0 = sv + (size_t)m * n_s + n;
  const float t00 = Elem<T>::get(r0), t01 = Elem<T>::get(r0 + 1);
  const float v0 = fmaf(fs, t01 - t00, t00);
  const float dv0 = t01 - t00;
  float v1, dv1;
  if (m + 1 < n_alpha) {
    const float t10 = Elem<T>::get(r0 + n_s), t11 = Elem<T>::get(r0 + n_s + 1);
    v1 = fmaf(fs, t11 - t10, t10);
    dv1 = t11 - t10;
  } else {  // row 0 at bins n_s - 1 - n and n_s - 2 - n
    const T* q = sv + (n_s - 2 - n);
    const float t10 = Elem<T>::get(q + 1), t11 = Elem<T>::get(q);
    v1 = -fmaf(fs, t11 - t10, t10);
    dv1 = -(t11 - t10);
  }
  const float Ba = (v1 - v0) * inv_dalpha * scale;
  const float Bs = fmaf(fa, dv1 - dv0, dv0) * inv_ds_f * scale;
  const float L0 = sign * l0, L1 = sign * l1, L2 = sign * l2;
  const float ih = rsqrtf(fmaf(L0, L0, L1 * L1));
  const float ca = L0 * ih, sa = L1 * ih, sf = -L2 * ih;
  g[0] = ih * (-Ba * sa - Bs * sf * ca);
  g[1] = ih * (Ba * ca - Bs * sf * sa);
  g[2] = -ih * Bs;
  return scale * sign * fmaf(fa, v1 - v0, v0);
}

// ------------------------------------------------------------ forward fast path
//
// The forward kernel takes tiles of 64 samples: each lane evaluates samples lane and
// lane + 32 of a tile from the tile's one anchor per view, so an anchor serves twice
// the samples of the 32-sample tiles of the adjoint, and one anchor pass (one anchor
// per lane) covers eight tiles of two pairs, which a warp evaluates one after the
// other.  A tile is evaluated with the anchors' own number of series terms
// (warp-uniform), without per-sample clamps and with two-row gathers at 32-bit
// indices.  A tile in which some lane's alpha row is outside [0, n_alpha - 2] (the
// fold at alpha = pi and the wrap of the last row) keeps these positions and samples
// them through the general gather with the fold applied (loc_folded); a tile in which
// a view needs the closed form is evaluated by the general per-sample code above.
// Positions are bitwise those of the general code (zero coefficients beyond the
// anchor's terms leave its Horner chains unchanged).  Launches with n_kappa below 96
// take the adjoint's kernel instead (kMinKappaForward64).

// Per-lane constants of one tile shape (adjoint: full tiles, or the ragged last tile).
struct LaneGeom {
  float jj, de, t, t2, tmd, cd, sd;
};

// Forward per-lane constants of one sample offset jj (sample steps from the anchor):
// t = tan(jj dk), t^2 and tan(jj dk) - jj dk.  The general code derives the rest.
struct LaneT {
  float jj, t, t2, tmd;
};

__device__ __forceinline__ LaneT lane_t(float jj, float dkf) {
  LaneT q;
  q.jj = jj;
  const float de = jj * dkf;
  q.t = tanf(de);
  q.t2 = q.t * q.t;
  q.tmd = tan_minus_angle(de, q.t);
  return q;
}

template <int NT, class Q>
__device__ __forceinline__ void series_position(const float4* __restrict__ rec, const Q& q, unsigned& mu,
                                                int& n, float& fa, float& fs) {
  const float4 h0 = rec[0], h1 = rec[1];
  const float* __restrict__ c = reinterpret_cast<const float*>(rec + 2);  // dco[kSer], sco[kSer]
  float da = c[NT - 1];
#pragma unroll
  for (int k = NT - 2; k >= 0; --k) da = fmaf(da, q.t, c[k]);
  da *= q.t;
  float sr = c[kSer + NT - 1];
#pragma unroll
  for (int k = NT - 2; k >= 1; --k) sr = fmaf(sr, q.t, c[kSer + k]);
  sr = fmaf(c[kSer], q.tmd, q.t2 * sr);
  const float lin = h1.y * q.jj;  // gh * jj: exact
  // floors and integer parts by one round-down add against M = 1.5 * 2^23 (float spacing
  // 1 in [2^23, 2^24)): RD(x + M) = M + floor(x) exactly for |x| < 2^22, and its bit
  // pattern minus that of M is floor(x) as an integer (no conversion instructions).
  // Masked lanes may carry larger values: their rows are rejected by the vote below.
  const float M = 12582912.0f;
  const float tl = __fadd_rd(lin, M);
  const float fa_ = h0.z + da;
  const float fs_ = (h0.w + (lin - (tl - M))) + fmaf(h1.z, q.jj, sr);
  const float ta = __fadd_rd(fa_, M), tn = __fadd_rd(fs_, M);
  mu = (unsigned)__float_as_int(h0.x) + (__float_as_uint(ta) - 0x4B400000u);
  n = (int)((unsigned)__float_as_int(h0.y) + (__float_as_uint(tl) - 0x4B400000u) + (__float_as_uint(tn) - 0x4B400000u));
  fa = fa_ - (ta - M);
  fs = fs_ - (tn - M);
}

// Bilinear value at row m (0 <= m <= n_alpha - 2) and bin n (clamped to [0, n_s - 2]);
// n_alpha n_s < 2^32, so the element index fits 32 bits.
template <typename T>
__device__ __forceinline__ float bilinear_rows(const T* __restrict__ sv, int n_s, unsigned m, int n, float fa,
                                               float fs) {
  n = min(max(n, 0), n_s - 2);
  const unsigned i0 = m * (unsigned)n_s + (unsigned)n;
  const T* __restrict__ r0 = sv + i0;
  const T* __restrict__ r1 = sv + (i0 + (unsigned)n_s);
  const float t00 = Elem<T>::get(r0), t01 = Elem<T>::get(r0 + 1);
  const float t10 = Elem<T>::get(r1), t11 = Elem<T>::get(r1 + 1);
  const float v0 = fmaf(fs, t01 - t00, t00);
  const float v1 = fmaf(fs, t11 - t10, t10);
  return fmaf(fa, v1 - v0, v0);
}

// The general code's Loc of a fast-path position (row mu as an unsigned sum, bin n,
// fractions): the fold of alpha into [0, pi) applied as loc_tail applies it.  For a
// tile in which some lane's row left [0, n_alpha - 2] (the fold at alpha = pi or the
// wrap of the last row): the positions are those of the general code, and so are
// the values sampled through it.
__device__ __forceinline__ Loc loc_folded(unsigned mu, int n, float fa, float fs, float sg, int n_alpha, int n_s) {
  Loc o;
  o.m = (int)mu;
  o.n = n;
  o.fa = fa;
  o.fs = fs;
  o.sign = sg;
  if (o.m >= n_alpha || o.m < 0) {  // S(alpha + pi, s) = -S(alpha, -s)
    o.m += o.m < 0 ? n_alpha : -n_alpha;
    o.n = n_s - 2 - o.n;
    o.fs = 1.0f - o.fs;
    o.sign = -o.sign;
  }
  o.ok = o.m >= 0 && o.m < n_alpha;  // false only for a masked sample
  return o;
}

// Difference S_a - S_b of one sample (offset jj from the anchors) by the general
// per-sample code: either evaluation, any alpha row (the fold and the wrap included).
template <typename T>
__device__ __noinline__ float sample_diff_general(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                                  float jj, float t, float tmd, float dkf, const T* __restrict__ sa,
                                                  const T* __restrict__ sb, float sca, float scb, int n_alpha,
                                                  int n_s, float inv_dalpha, float inv_ds_f) {
  const float de = jj * dkf;
  float sd, cd;
  sincosf(de, &sd, &cd);
  Loc la, lb;
  {
    const Anchor an = load_anchor(ra);
    la = an.ser != 0.0f ? locate_series(an, t, tmd, jj, n_alpha, n_s)
                        : locate(an, cd, sd, jj, de, n_alpha, n_s, inv_dalpha, inv_ds_f);
  }
  {
    const Anchor an = load_anchor(rb);
    lb = an.ser != 0.0f ? locate_series(an, t, tmd, jj, n_alpha, n_s)
                        : locate(an, cd, sd, jj, de, n_alpha, n_s, inv_dalpha, inv_ds_f);
  }
  return sca * sample(sa, n_alpha, n_s, la) - scb * sample(sb, n_alpha, n_s, lb);
}

// One sample per lane (a last tile of at most 32 samples).
template <typename T, int NT>
__device__ __forceinline__ float sample_diff_series(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                                   const LaneT& q, float dkf, const T* __restrict__ sa,
                                                   const T* __restrict__ sb, float sca, float scb, int n_alpha,
                                                   int n_s, float inv_dalpha, float inv_ds_f) {
  unsigned ma, mb;
  int na, nb;
  float faa, fsa, fab, fsb;
  series_position<NT>(ra, q, ma, na, faa, fsa);
  series_position<NT>(rb, q, mb, nb, fab, fsb);
  const unsigned last = (unsigned)(n_alpha - 1);
  if (__any_sync(0xffffffffu, ma >= last || mb >= last))  // fold or last-row wrap somewhere in the tile
    return sca * sample(sa, n_alpha, n_s, loc_folded(ma, na, faa, fsa, ra[1].x, n_alpha, n_s)) -
           scb * sample(sb, n_alpha, n_s, loc_folded(mb, nb, fab, fsb, rb[1].x, n_alpha, n_s));
  const float ga = sca * ra[1].x, gb = scb * rb[1].x;  // storage scale times the anchor's fold
  return ga * bilinear_rows(sa, n_s, ma, na, faa, fsa) - gb * bilinear_rows(sb, n_s, mb, nb, fab, fsb);
}

template <typename T>
__device__ __forceinline__ float sample_diff(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                            const LaneT& q, float dkf, const T* __restrict__ sa,
                                            const T* __restrict__ sb, float sca, float scb, int n_alpha, int n_s,
                                            float inv_dalpha, float inv_ds_f) {
  const float na = ra[1].w, nb = rb[1].w;  // terms of the two anchors (warp-uniform)
  if (na == 0.0f || nb == 0.0f)
    return sample_diff_general<T>(ra, rb, q.jj, q.t, q.tmd, dkf, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha,
                                  inv_ds_f);
  const float nt = fmaxf(na, nb);
#define ECC_ONE(NT_) \
  return sample_diff_series<T, NT_>(ra, rb, q, dkf, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha, inv_ds_f)
  if (nt <= 3.0f) ECC_ONE(3);
  if (nt <= 4.0f) ECC_ONE(4);
  if (nt <= 6.0f) ECC_ONE(6);
  if (nt <= 8.0f) ECC_ONE(8);
  if (nt <= 12.0f) ECC_ONE(12);
  ECC_ONE(kSer);
#undef ECC_ONE
}

// Both samples of every lane in a tile (offsets q0 and q1 from the same anchors).
template <typename T, int NT>
__device__ __forceinline__ bool tile_diff_series(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                                 const LaneT& q0, const LaneT& q1, const T* __restrict__ sa,
                                                 const T* __restrict__ sb, float sca, float scb, int n_alpha,
                                                 int n_s, float& d0, float& d1) {
  unsigned ma0, mb0, ma1, mb1;
  int na0, nb0, na1, nb1;
  float fa0, fs0, fb0, gs0, fa1, fs1, fb1, gs1;
  series_position<NT>(ra, q0, ma0, na0, fa0, fs0);
  series_position<NT>(ra, q1, ma1, na1, fa1, fs1);
  series_position<NT>(rb, q0, mb0, nb0, fb0, gs0);
  series_position<NT>(rb, q1, mb1, nb1, fb1, gs1);
  const unsigned last = (unsigned)(n_alpha - 1);
  if (__any_sync(0xffffffffu, ma0 >= last || mb0 >= last || ma1 >= last || mb1 >= last)) {
    d0 = sca * sample(sa, n_alpha, n_s, loc_folded(ma0, na0, fa0, fs0, ra[1].x, n_alpha, n_s)) -
         scb * sample(sb, n_alpha, n_s, loc_folded(mb0, nb0, fb0, gs0, rb[1].x, n_alpha, n_s));
    d1 = sca * sample(sa, n_alpha, n_s, loc_folded(ma1, na1, fa1, fs1, ra[1].x, n_alpha, n_s)) -
         scb * sample(sb, n_alpha, n_s, loc_folded(mb1, nb1, fb1, gs1, rb[1].x, n_alpha, n_s));
    return true;
  }
  const float ga = sca * ra[1].x, gb = scb * rb[1].x;
  const float A0 = bilinear_rows(sa, n_s, ma0, na0, fa0, fs0), B0 = bilinear_rows(sb, n_s, mb0, nb0, fb0, gs0);
  const float A1 = bilinear_rows(sa, n_s, ma1, na1, fa1, fs1), B1 = bilinear_rows(sb, n_s, mb1, nb1, fb1, gs1);
  d0 = ga * A0 - gb * B0;
  d1 = ga * A1 - gb * B1;
  return true;
}

template <typename T>
__device__ __forceinline__ void tile_diff(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                          const LaneT& q0, const LaneT& q1, float dkf, const T* __restrict__ sa,
                                          const T* __restrict__ sb, float sca, float scb, int n_alpha, int n_s,
                                          float inv_dalpha, float inv_ds_f, float& d0, float& d1) {
  const float na = ra[1].w, nb = rb[1].w;  // terms of the two anchors (warp-uniform)
  bool done = false;
  if (na != 0.0f && nb != 0.0f) {
    const float nt = fmaxf(na, nb);
#define ECC_TWO(NT_) tile_diff_series<T, NT_>(ra, rb, q0, q1, sa, sb, sca, scb, n_alpha, n_s, d0, d1)
    if (nt <= 3.0f)
      done = ECC_TWO(3);
    else if (nt <= 4.0f)
      done = ECC_TWO(4);
    else if (nt <= 6.0f)
      done = ECC_TWO(6);
    else if (nt <= 8.0f)
      done = ECC_TWO(8);
    else if (nt <= 12.0f)
      done = ECC_TWO(12);
    else
      done = ECC_TWO(kSer);
#undef ECC_TWO
  }
  if (!done) {
    d0 = sample_diff_general<T>(ra, rb, q0.jj, q0.t, q0.tmd, dkf, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha,
                                inv_ds_f);
    d1 = sample_diff_general<T>(ra, rb, q1.jj, q1.t, q1.tmd, dkf, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha,
                                inv_ds_f);
  }
}

// Forward values of pairs p0 and (if has1) p1 on one warp: d (Eq. 15), the Cauchy e
// (Eq. 16) and N_kappa of each; returns the sum of their e.  Tiles of 64 samples; the
// anchor pass takes lane = 16 (pair) + 8 (view) + tile, eight tiles of both pairs.
// A tile's anchor sits at the sum of its two 32-sample centre directions, which is
// the direction of their mean angle (the anchor depends on the direction only, not
// on its length): the tile's centre for full tiles; for a last tile of 33..63
// samples the mean of the two centres, within 31.5 steps of each of its samples.  A
// last tile of at most 32 samples is its own 32-sample tile.
template <typename T>
__device__ __forceinline__ double pair_warp2_forward(const PairArgs& g, long long p0, long long p1, bool has1,
                                                     int lane, float4* __restrict__ recw) {
  if (!has1) p1 = p0;  // the second half of the anchor pass repeats the first pair
  const int n_tiles = g.n_tiles, n_alpha = g.n_alpha, n_s = g.n_s, K = g.K;
  const int n_t64 = (K + 63) / 64;         // tiles of 64 samples (n_tiles counts those of 32)
  const int n_rem = K - 64 * (n_t64 - 1);  // samples of the last one (1 .. 64)
  const int nk0 = g.prs[p0].status == 0 ? g.prs[p0].nk : 0;
  const int nk1 = has1 && g.prs[p1].status == 0 ? g.prs[p1].nk : 0;
  const float inv_dalpha = g.inv_dalpha, inv_ds_f = g.inv_ds_f;
  float acc0 = 0.0f, acc1 = 0.0f;
  if (nk0 > 0 || nk1 > 0) {
    const T* __restrict__ sino = static_cast<const T*>(g.sino);
    const size_t vstride = (size_t)n_alpha * n_s;
    for (int t0 = 0; t0 < n_t64; t0 += 8) {
      {
        const long long p = (lane >> 4) ? p1 : p0;
        const PairRec& pr = g.prs[p];
        const int v = (lane >> 3) & 1;
        const int u = min(t0 + (lane & 7), n_t64 - 1);
        const float4* __restrict__ ct = g.ctile + p * n_tiles;
        float4 c = ct[2 * u];
        if (2 * u + 1 < n_tiles) {
          const float4 cb = ct[2 * u + 1];
          const df x = df_add(df{c.x, c.z}, df{cb.x, cb.z}), y = df_add(df{c.y, c.w}, df{cb.y, cb.w});
          c = make_float4(x.hi, y.hi, x.lo, y.lo);
        }
        const df inv_ds = {g.inv_ds_hi, g.inv_ds_lo};
        const df half_ns1 = {g.half_hi, g.half_lo};
        const df dk = {pr.dk_hi, pr.dk_lo};
        store_anchor(recw + kRec * lane, make_anchor(pr.Af[v], c, g.alpha_dir, n_alpha, inv_dalpha, inv_ds, half_ns1,
                                                  inv_ds_f, dk, tanf(31.5f * pr.dk_hi), kGhMask64, kSerLimit64, kSer));
      }
      __syncwarp();
      const int umax = min(8, n_t64 - t0);
      const int ufull = (t0 + umax == n_t64 && n_rem != 64) ? umax - 1 : umax;
#pragma unroll 1
      for (int ps = 0; ps < 2; ++ps) {
        if ((ps ? nk1 : nk0) == 0) continue;  // warp-uniform
        const PairRec& pr = g.prs[ps ? p1 : p0];
        const T* __restrict__ sa = sino + (size_t)pr.a * vstride;
        const T* __restrict__ sb = sino + (size_t)pr.b * vstride;
        const float sca = g.scales ? g.scales[pr.a] : 1.0f;
        const float scb = g.scales ? g.scales[pr.b] : 1.0f;
        const float dkf = pr.dk_hi;
        unsigned vm = 0;  // bit 2 uu + h: sample 64 (t0 + uu) + 32 h + lane is valid
        {
          const int r0lo = pr.r0lo, r1lo = pr.r1lo;
          const unsigned len0 = (unsigned)max(pr.r0hi - pr.r0lo, 0), len1 = (unsigned)max(pr.r1hi - pr.r1lo, 0);
#pragma unroll
          for (int bit = 0; bit < 16; ++bit) {
            const int k = 64 * t0 + 32 * bit + lane;
            if (k < K && ((unsigned)(k - r0lo) < len0 || (unsigned)(k - r1lo) < len1)) vm |= 1u << bit;
          }
        }
        const float4* __restrict__ rw = recw + kRec * 16 * ps;  // view a: tiles 0..7, view b: tiles 8..15
        float acc = 0.0f;
        if (ufull > 0) {
          const LaneT q0 = lane_t((float)lane - 31.5f, dkf), q1 = lane_t((float)lane + 0.5f, dkf);
          for (int uu = 0; uu < ufull; ++uu) {
            float d0, d1;
            tile_diff<T>(rw + kRec * uu, rw + kRec * (8 + uu), q0, q1, dkf, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha,
                         inv_ds_f, d0, d1);
            acc += (vm >> (2 * uu)) & 1u ? d0 * d0 : 0.0f;
            acc += (vm >> (2 * uu + 1)) & 1u ? d1 * d1 : 0.0f;
          }
        }
        if (ufull < umax) {  // the ragged last tile
          const float4* __restrict__ ra = rw + kRec * ufull;
          const float4* __restrict__ rb = rw + kRec * (8 + ufull);
          if (n_rem > 32) {
            const float mid = 15.5f + 0.25f * (float)n_rem;  // anchor: mean angle of the two 32-sample centres
            float d0, d1;
            tile_diff<T>(ra, rb, lane_t((float)lane - mid, dkf), lane_t((float)lane + 32.0f - mid, dkf), dkf, sa, sb,
                         sca, scb, n_alpha, n_s, inv_dalpha, inv_ds_f, d0, d1);
            acc += (vm >> (2 * ufull)) & 1u ? d0 * d0 : 0.0f;
            acc += (vm >> (2 * ufull + 1)) & 1u ? d1 * d1 : 0.0f;
          } else {
            const float dd = sample_diff<T>(ra, rb, lane_t((float)lane + 0.5f - 0.5f * (float)n_rem, dkf), dkf, sa,
                                            sb, sca, scb, n_alpha, n_s, inv_dalpha, inv_ds_f);
            acc += (vm >> (2 * ufull)) & 1u ? dd * dd : 0.0f;
          }
        }
        if (ps)
          acc1 += acc;
        else
          acc0 += acc;
      }
      __syncwarp();  // records are rewritten by the next chunk
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
    acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
  }
  double e_sum = 0.0;
  for (int ps = 0; ps < (has1 ? 2 : 1); ++ps) {
    const long long p = ps ? p1 : p0;
    const float acc = ps ? acc1 : acc0;
    // a non-finite sum (non-finite sinogram values) drops the pair: N_kappa = 0, d = e = 0
    const bool finite = isfinite(acc);
    const int nk = finite ? (ps ? nk1 : nk0) : 0;
    const float d = nk > 0 ? acc / (float)nk : 0.0f;
    const float e = g.cauchy_c > 0.0f ? d / (1.0f + d / g.cauchy_c) : d;
    if (lane == 0) {
      if (!finite && g.status) atomicOr(g.status, kStatusNonfinitePair);
      if (g.per_pair) {
        g.per_pair[2 * p] = (double)d;
        g.per_pair[2 * p + 1] = (double)e;
      }
      if (g.nk_out) g.nk_out[p] = nk;
    }
    e_sum += (double)e;
  }
  return e_sum;
}

// ------------------------------------------------------------ adjoint fast path
//
// The adjoint kernel uses the forward kernel's positions (series_position) and warp
// vote; the value and line gradient of a sample are those of sample_grad, written
// for a row in [0, n_alpha - 2] and the anchor's fold.

template <typename T>
__device__ __forceinline__ float sample_grad_rows(const T* __restrict__ sv, int n_s, unsigned m, int n, float fa,
                                                  float fs, float sign, float inv_dalpha, float inv_ds_f, float l0,
                                                  float l1, float l2, float scale, float (&g)[3]) {
  n = min(max(n, 0), n_s - 2);
  const unsigned i0 = m * (unsigned)n_s + (unsigned)n;
  const T* __restrict__ r0 = sv + i0;
  const T* __restrict__ r1 = sv + (i0 + (unsigned)n_s);
  const float t00 = Elem<T>::get(r0), t01 = Elem<T>::get(r0 + 1);
  const float t10 = Elem<T>::get(r1), t11 = Elem<T>::get(r1 + 1);
  const float dv0 = t01 - t00, dv1 = t11 - t10;
  const float v0 = fmaf(fs, dv0, t00), v1 = fmaf(fs, dv1, t10);
  const float Ba = (v1 - v0) * inv_dalpha * scale;
  const float Bs = fmaf(fa, dv1 - dv0, dv0) * inv_ds_f * scale;
  const float L0 = sign * l0, L1 = sign * l1, L2 = sign * l2;
  const float ih = rsqrtf(fmaf(L0, L0, L1 * L1));
  const float ca = L0 * ih, sa = L1 * ih, sf = -L2 * ih;
  g[0] = ih * (-Ba * sa - Bs * sf * ca);
  g[1] = ih * (Ba * ca - Bs * sf * sa);
  g[2] = -ih * Bs;
  return scale * sign * fmaf(fa, v1 - v0, v0);
}

// The lane's line l = A c_k of one view from its tile's record (written by the anchor
// pass): c_k = cos(delta) c_t + sin(delta) c_t_perp, so l = cos(delta) (A c_t) + sin(delta)
// (A c_t_perp), with A c_t = (x.x, x.y, x.z) and A c_t_perp = (x.w, y.x, y.y).
__device__ __forceinline__ void tile_line(const float4* __restrict__ lp, float cd, float sd, float& l0, float& l1,
                                          float& l2) {
  const float4 x = lp[0], y = lp[1];
  l0 = fmaf(sd, x.w, cd * x.x);
  l1 = fmaf(sd, y.x, cd * x.y);
  l2 = fmaf(sd, y.y, cd * x.z);
}

// S_a - S_b of this lane's sample and the line gradients of both views, by the general
// per-sample code.
template <typename T>
__device__ __forceinline__ float tile_adjoint_general_body(const float4* __restrict__ ra,
                                                          const float4* __restrict__ rb, const LaneGeom& q,
                                                          const T* __restrict__ sa, const T* __restrict__ sb,
                                                          float sca, float scb, int n_alpha, int n_s,
                                                          float inv_dalpha, float inv_ds_f,
                                                          const float4* __restrict__ lpa,
                                                          const float4* __restrict__ lpb, float (&ga)[3],
                                                          float (&gb)[3]) {
  Loc la, lb;
  {
    const Anchor an = load_anchor(ra);
    la = an.ser != 0.0f ? locate_series(an, q.t, q.tmd, q.jj, n_alpha, n_s)
                        : locate(an, q.cd, q.sd, q.jj, q.de, n_alpha, n_s, inv_dalpha, inv_ds_f);
  }
  {
    const Anchor an = load_anchor(rb);
    lb = an.ser != 0.0f ? locate_series(an, q.t, q.tmd, q.jj, n_alpha, n_s)
                        : locate(an, q.cd, q.sd, q.jj, q.de, n_alpha, n_s, inv_dalpha, inv_ds_f);
  }
  float l0, l1, l2;
  tile_line(lpa, q.cd, q.sd, l0, l1, l2);
  const float Sa = sample_grad(sa, n_alpha, n_s, la, inv_dalpha, inv_ds_f, l0, l1, l2, sca, ga);
  tile_line(lpb, q.cd, q.sd, l0, l1, l2);
  const float Sb = sample_grad(sb, n_alpha, n_s, lb, inv_dalpha, inv_ds_f, l0, l1, l2, scb, gb);
  return Sa - Sb;
}

template <typename T>
__device__ __noinline__ float tile_adjoint_general(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                                  const LaneGeom& q, const T* __restrict__ sa,
                                                  const T* __restrict__ sb, float sca, float scb, int n_alpha,
                                                  int n_s, float inv_dalpha, float inv_ds_f,
                                                  const float4* __restrict__ lpa, const float4* __restrict__ lpb,
                                                  float (&ga)[3], float (&gb)[3]) {
  return tile_adjoint_general_body<T>(ra, rb, q, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha, inv_ds_f, lpa, lpb, ga,
                                      gb);
}

template <typename T, int NT>
__device__ __forceinline__ float tile_adjoint_series(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                                    const LaneGeom& q, const T* __restrict__ sa,
                                                    const T* __restrict__ sb, float sca, float scb, int n_alpha,
                                                    int n_s, float inv_dalpha, float inv_ds_f,
                                                    const float4* __restrict__ lpa,
                                                    const float4* __restrict__ lpb, float (&ga)[3], float (&gb)[3]) {
  unsigned ma, mb;
  int na, nb;
  float faa, fsa, fab, fsb;
  series_position<NT>(ra, q, ma, na, faa, fsa);
  series_position<NT>(rb, q, mb, nb, fab, fsb);
  const unsigned last = (unsigned)(n_alpha - 1);
  if (__any_sync(0xffffffffu, ma >= last || mb >= last))
    return tile_adjoint_general<T>(ra, rb, q, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha, inv_ds_f, lpa, lpb, ga,
                                   gb);
  float l0, l1, l2;
  tile_line(lpa, q.cd, q.sd, l0, l1, l2);
  const float Sa = sample_grad_rows(sa, n_s, ma, na, faa, fsa, ra[1].x, inv_dalpha, inv_ds_f, l0, l1, l2, sca, ga);
  tile_line(lpb, q.cd, q.sd, l0, l1, l2);
  const float Sb = sample_grad_rows(sb, n_s, mb, nb, fab, fsb, rb[1].x, inv_dalpha, inv_ds_f, l0, l1, l2, scb, gb);
  return Sa - Sb;
}

// Two tiles at once (the lane's samples of tiles u and u + 1, offsets q from the anchors
// of each): positions of all four view-samples first, then all sixteen taps, so that the
// gathers of both tiles are in flight together.  Returns false, with nothing computed, if
// some lane's row leaves [0, n_alpha - 2] in either tile (the caller then takes the
// tiles one at a time).
template <typename T, int NT>
__device__ __forceinline__ bool tile_adjoint_series2(const float4* __restrict__ ra0, const float4* __restrict__ rb0,
                                                     const float4* __restrict__ ra1, const float4* __restrict__ rb1,
                                                     const LaneGeom& q, const T* __restrict__ sa,
                                                     const T* __restrict__ sb, float sca, float scb, int n_alpha,
                                                     int n_s, float inv_dalpha, float inv_ds_f,
                                                     const float4* __restrict__ lpa0, const float4* __restrict__ lpb0,
                                                     const float4* __restrict__ lpa1, const float4* __restrict__ lpb1,
                                                     float& dd0, float (&ga0)[3], float (&gb0)[3], float& dd1,
                                                     float (&ga1)[3], float (&gb1)[3]) {
  unsigned ma0, mb0, ma1, mb1;
  int na0, nb0, na1, nb1;
  float fa0, fs0, fb0, gs0, fa1, fs1, fb1, gs1;
  series_position<NT>(ra0, q, ma0, na0, fa0, fs0);
  series_position<NT>(rb0, q, mb0, nb0, fb0, gs0);
  series_position<NT>(ra1, q, ma1, na1, fa1, fs1);
  series_position<NT>(rb1, q, mb1, nb1, fb1, gs1);
  const unsigned last = (unsigned)(n_alpha - 1);
  if (__any_sync(0xffffffffu, ma0 >= last || mb0 >= last || ma1 >= last || mb1 >= last)) return false;
  float l0, l1, l2;
  tile_line(lpa0, q.cd, q.sd, l0, l1, l2);
  const float Sa0 = sample_grad_rows(sa, n_s, ma0, na0, fa0, fs0, ra0[1].x, inv_dalpha, inv_ds_f, l0, l1, l2, sca, ga0);
  tile_line(lpb0, q.cd, q.sd, l0, l1, l2);
  const float Sb0 = sample_grad_rows(sb, n_s, mb0, nb0, fb0, gs0, rb0[1].x, inv_dalpha, inv_ds_f, l0, l1, l2, scb, gb0);
  tile_line(lpa1, q.cd, q.sd, l0, l1, l2);
  const float Sa1 = sample_grad_rows(sa, n_s, ma1, na1, fa1, fs1, ra1[1].x, inv_dalpha, inv_ds_f, l0, l1, l2, sca, ga1);
  tile_line(lpb1, q.cd, q.sd, l0, l1, l2);
  const float Sb1 = sample_grad_rows(sb, n_s, mb1, nb1, fb1, gs1, rb1[1].x, inv_dalpha, inv_ds_f, l0, l1, l2, scb, gb1);
  dd0 = Sa0 - Sb0;
  dd1 = Sa1 - Sb1;
  return true;
}

template <typename T>
__device__ __forceinline__ bool tile_adjoint2(const float4* __restrict__ ra0, const float4* __restrict__ rb0,
                                              const float4* __restrict__ ra1, const float4* __restrict__ rb1,
                                              const LaneGeom& q, const T* __restrict__ sa, const T* __restrict__ sb,
                                              float sca, float scb, int n_alpha, int n_s, float inv_dalpha,
                                              float inv_ds_f, const float4* __restrict__ lpa0,
                                              const float4* __restrict__ lpb0, const float4* __restrict__ lpa1,
                                              const float4* __restrict__ lpb1, float& dd0, float (&ga0)[3],
                                              float (&gb0)[3], float& dd1, float (&ga1)[3], float (&gb1)[3]) {
  const float n0 = ra0[1].w, n1 = rb0[1].w, n2 = ra1[1].w, n3 = rb1[1].w;
  if (n0 == 0.0f || n1 == 0.0f || n2 == 0.0f || n3 == 0.0f) return false;  // a closed-form anchor
  const float nt = fmaxf(fmaxf(n0, n1), fmaxf(n2, n3));
#define ECC_ADJ2(NT_)                                                                                          \
  return tile_adjoint_series2<T, NT_>(ra0, rb0, ra1, rb1, q, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha,        \
                                      inv_ds_f, lpa0, lpb0, lpa1, lpb1, dd0, ga0, gb0, dd1, ga1, gb1)
  if (nt <= 3.0f) ECC_ADJ2(3);
  if (nt <= 4.0f) ECC_ADJ2(4);
  if (nt <= 6.0f) ECC_ADJ2(6);
  if (nt <= 8.0f) ECC_ADJ2(8);
  ECC_ADJ2(12);
#undef ECC_ADJ2
}

template <typename T>
__device__ __forceinline__ float tile_adjoint(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                             const LaneGeom& q, const T* __restrict__ sa, const T* __restrict__ sb,
                                             float sca, float scb, int n_alpha, int n_s, float inv_dalpha,
                                             float inv_ds_f, const float4* __restrict__ lpa,
                                             const float4* __restrict__ lpb, float (&ga)[3], float (&gb)[3]) {
  const float na = ra[1].w, nb = rb[1].w;
  if (na == 0.0f || nb == 0.0f)
    return tile_adjoint_general<T>(ra, rb, q, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha, inv_ds_f, lpa, lpb, ga, gb);
  const float nt = fmaxf(na, nb);
#define ECC_ADJ(NT_) \
  return tile_adjoint_series<T, NT_>(ra, rb, q, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha, inv_ds_f, lpa, lpb, ga, gb)
  if (nt <= 3.0f) ECC_ADJ(3);
  if (nt <= 4.0f) ECC_ADJ(4);
  if (nt <= 6.0f) ECC_ADJ(6);
  if (nt <= 8.0f) ECC_ADJ(8);
  if (nt <= 12.0f) ECC_ADJ(12);
  ECC_ADJ(kSer);
#undef ECC_ADJ
}

// Adjoint of pair p on one warp: d, e, N_kappa as the forward kernel, and d e / d A
// (de/dd)/N_kappa sum_k 2 (S_a - S_b) (dS/dl) c_k^T for the gradient kernels.
// FAST: tiles dispatch on the anchors' term counts (the single-scan kernel); otherwise
// every tile takes the general per-sample code inline (the persistent serving kernel,
// whose three storage types would otherwise carry fifteen tile variants; same positions
// and formulas, so the same values).
template <typename T, bool FAST>
__device__ __forceinline__ double pair_warp_adjoint(const PairArgs& g, long long p, int lane,
                                                    float4* __restrict__ recw, float4* __restrict__ lpw) {
  const PairRec& pr = g.prs[p];
  const int nk_in = pr.status == 0 ? pr.nk : 0;
  const int n_tiles = g.n_tiles, n_alpha = g.n_alpha, n_s = g.n_s, K = g.K;
  float acc = 0.0f;
  float G[12];  // sum_k 2 (S_a - S_b) (dS/dl) c_k^T for views a (0..5), b (6..11)
#pragma unroll
  for (int i = 0; i < 12; ++i) G[i] = 0.0f;
  if (nk_in > 0) {
    const T* __restrict__ sino = static_cast<const T*>(g.sino);
    const size_t vstride = (size_t)n_alpha * n_s;
    const T* __restrict__ sa = sino + (size_t)pr.a * vstride;
    const T* __restrict__ sb = sino + (size_t)pr.b * vstride;
    const float sca = g.scales ? g.scales[pr.a] : 1.0f;
    const float scb = g.scales ? g.scales[pr.b] : 1.0f;
    const float inv_dalpha = g.inv_dalpha, inv_ds_f = g.inv_ds_f;
    const df inv_ds = {g.inv_ds_hi, g.inv_ds_lo};
    const df half_ns1 = {g.half_hi, g.half_lo};
    const float dkf = pr.dk_hi;
    const df dk = {pr.dk_hi, pr.dk_lo};
    auto lane_geom = [&](float jj) {
      LaneGeom q;
      q.jj = jj;
      q.de = jj * dkf;
      sincosf(q.de, &q.sd, &q.cd);
      q.t = tanf(q.de);
      q.t2 = q.t * q.t;
      q.tmd = tan_minus_angle(q.de, q.t);
      return q;
    };
    const int n_last = K - 32 * (n_tiles - 1);
    const LaneGeom qf = lane_geom((float)lane - 15.5f);
    const float jj_last = (float)lane + 0.5f - 0.5f * (float)n_last;  // the ragged tile's offsets
    const float tan_half_tile = tanf(15.5f * dkf);
    const int r0lo = pr.r0lo, r1lo = pr.r1lo;
    const unsigned len0 = (unsigned)max(pr.r0hi - pr.r0lo, 0), len1 = (unsigned)max(pr.r1hi - pr.r1lo, 0);
    const float4* __restrict__ ct = g.ctile + p * n_tiles;
    auto one_tile = [&](int t, const LaneGeom& q, bool valid) {
      const float4 ctd = ct[t];
      const float ckx = ctd.x * q.cd - ctd.y * q.sd, cky = ctd.x * q.sd + ctd.y * q.cd;
      float ga[3], gb[3];
      const int tt = t & 15;
      const float dd =
          FAST ? tile_adjoint<T>(recw + kRec * tt, recw + kRec * (16 + tt), q, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha,
                                 inv_ds_f, lpw + 2 * tt, lpw + 2 * (16 + tt), ga, gb)
               : tile_adjoint_general_body<T>(recw + kRec * tt, recw + kRec * (16 + tt), q, sa, sb, sca, scb, n_alpha,
                                              n_s, inv_dalpha, inv_ds_f, lpw + 2 * tt, lpw + 2 * (16 + tt), ga, gb);
      acc += valid ? dd * dd : 0.0f;
      // masked samples may sit anywhere (their slopes need not be finite): skipped, not
      // multiplied by zero
      if (valid) {
        const float w2 = 2.0f * dd;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          G[2 * i] = fmaf(w2 * ga[i], ckx, G[2 * i]);
          G[2 * i + 1] = fmaf(w2 * ga[i], cky, G[2 * i + 1]);
          G[6 + 2 * i] = fmaf(-w2 * gb[i], ckx, G[6 + 2 * i]);
          G[6 + 2 * i + 1] = fmaf(-w2 * gb[i], cky, G[6 + 2 * i + 1]);
        }
      }
    };
    for (int t0 = 0; t0 < n_tiles; t0 += 16) {
      {
        const int v = lane >> 4;
        int t = t0 + (lane & 15);
        if (t >= n_tiles) t = n_tiles - 1;
        const float4 c = ct[t];
        store_anchor(recw + kRec * lane, make_anchor(pr.Af[v], c, g.alpha_dir, n_alpha, inv_dalpha, inv_ds,
                                                  half_ns1, inv_ds_f, dk, tan_half_tile, kGhMask32, kSerLimit32, 10));
        // the tile's lines A c_t and A c_t_perp (FP32) for the per-sample line gradients
        const float* A = pr.Af[v];  // (hi, lo) pairs: A[4 i] = row i, column 0; A[4 i + 2] = column 1
        float lc[3], pc[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          lc[i] = fmaf(A[4 * i + 2], c.y, A[4 * i] * c.x);
          pc[i] = fmaf(A[4 * i + 2], c.x, -A[4 * i] * c.y);
        }
        lpw[2 * lane] = make_float4(lc[0], lc[1], lc[2], pc[0]);
        lpw[2 * lane + 1] = make_float4(pc[1], pc[2], 0.0f, 0.0f);
      }
      __syncwarp();
      const int tmax = min(16, n_tiles - t0);
      const int tfull = (t0 + tmax == n_tiles && n_last != 32) ? tmax - 1 : tmax;
      int tt = 0;
      if (FAST) {
        // two full tiles per iteration: their gathers are in flight together
        for (; tt + 1 < tfull; tt += 2) {
          const int t = t0 + tt;
          float dd0, dd1, ga0[3], gb0[3], ga1[3], gb1[3];
          if (!tile_adjoint2<T>(recw + kRec * tt, recw + kRec * (16 + tt), recw + kRec * (tt + 1),
                                recw + kRec * (17 + tt), qf, sa, sb, sca, scb, n_alpha, n_s, inv_dalpha, inv_ds_f,
                                lpw + 2 * tt, lpw + 2 * (16 + tt), lpw + 2 * (tt + 1), lpw + 2 * (17 + tt), dd0, ga0,
                                gb0, dd1, ga1, gb1)) {
            for (int u = 0; u < 2; ++u) {
              const int k = 32 * (t + u) + lane;
              one_tile(t + u, qf, (unsigned)(k - r0lo) < len0 || (unsigned)(k - r1lo) < len1);
            }
            continue;
          }
          for (int u = 0; u < 2; ++u) {
            const int k = 32 * (t + u) + lane;
            const bool valid = (unsigned)(k - r0lo) < len0 || (unsigned)(k - r1lo) < len1;
            const float4 ctd = ct[t + u];
            const float ckx = ctd.x * qf.cd - ctd.y * qf.sd, cky = ctd.x * qf.sd + ctd.y * qf.cd;
            const float dd = u ? dd1 : dd0;
            acc += valid ? dd * dd : 0.0f;
            if (valid) {
              const float w2 = 2.0f * dd;
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                const float a = u ? ga1[i] : ga0[i], b = u ? gb1[i] : gb0[i];
                G[2 * i] = fmaf(w2 * a, ckx, G[2 * i]);
                G[2 * i + 1] = fmaf(w2 * a, cky, G[2 * i + 1]);
                G[6 + 2 * i] = fmaf(-w2 * b, ckx, G[6 + 2 * i]);
                G[6 + 2 * i + 1] = fmaf(-w2 * b, cky, G[6 + 2 * i + 1]);
              }
            }
          }
        }
      }
      for (; tt < tfull; ++tt) {
        const int k = 32 * (t0 + tt) + lane;
        one_tile(t0 + tt, qf, (unsigned)(k - r0lo) < len0 || (unsigned)(k - r1lo) < len1);
      }
      if (tfull < tmax) {
        const int k = 32 * (t0 + tfull) + lane;
        one_tile(t0 + tfull, lane_geom(jj_last),
                 k < K && ((unsigned)(k - r0lo) < len0 || (unsigned)(k - r1lo) < len1));
      }
      __syncwarp();
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
#pragma unroll
  for (int i = 0; i < 12; ++i)
    for (int o = 16; o > 0; o >>= 1) G[i] += __shfl_xor_sync(0xffffffffu, G[i], o);
  // a non-finite sum or gradient (non-finite sinogram values) drops the pair:
  // N_kappa = 0, d = e = 0 and no gradient
  bool finite = isfinite(acc);
#pragma unroll
  for (int i = 0; i < 12; ++i) finite = finite && isfinite(G[i]);
  const int nk = finite ? nk_in : 0;
  const float d = nk > 0 ? acc / (float)nk : 0.0f;
  const float e = g.cauchy_c > 0.0f ? d / (1.0f + d / g.cauchy_c) : d;
  if (lane == 0) {
    if (!finite && g.status) atomicOr(g.status, kStatusNonfinitePair);
    if (g.per_pair) {
      g.per_pair[2 * p] = (double)d;
      g.per_pair[2 * p + 1] = (double)e;
    }
    if (g.nk_out) g.nk_out[p] = nk;
    // d e / d A = (de/dd) (1/N) G
    const float r = g.cauchy_c > 0.0f ? 1.0f / (1.0f + d / g.cauchy_c) : 1.0f;
    const float scale = nk > 0 ? r * r / (float)nk : 0.0f;
    if (g.Gpp) {  // NULL: a forward evaluation through this code (small n_kappa)
#pragma unroll
      for (int i = 0; i < 12; ++i) g.Gpp[12 * p + i] = nk > 0 ? (double)(G[i] * scale) : 0.0;
    }
  }
  return (double)e;
}

// One block of consecutive pairs (kWarpsPerBlock for the adjoint, two per warp for the
// forward kernel): their e summed in a fixed order into partial[blk].
template <typename T, bool GRAD, bool SERVE = false>
__device__ __forceinline__ void pair_block(const PairArgs& g, long long blk, double* e_warp, float4* recs,
                                           float4* lps) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float4* recw = recs + (size_t)wib * 32 * kRec;
  double e_val = 0.0;
  if (GRAD) {
    const long long p = blk * kWarpsPerBlock + wib;
    if (p < g.n_pairs) e_val = pair_warp_adjoint<T, !SERVE>(g, p, lane, recw, lps + (size_t)wib * 64);  // warp-uniform
  } else {
    // two pairs per warp (blk 2W + w and blk 2W + W + w, W warps: the block's warps run
    // neighbouring pairs side by side) when the launch has fewer blocks than pairs / W
    const bool two = (long long)gridDim.x * kWarpsPerBlock < g.n_pairs;
    const long long p = blk * (two ? kPairsPerForwardBlock : kWarpsPerBlock) + wib;
    if (p < g.n_pairs)  // warp-uniform
      e_val = pair_warp2_forward<T>(g, p, p + kWarpsPerBlock, two && p + kWarpsPerBlock < g.n_pairs, lane, recw);
  }
  if (lane == 0) e_warp[wib] = e_val;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kWarpsPerBlock; ++w) s += e_warp[w];
    g.block_partial[blk] = s;
  }
  __syncthreads();
}

// The forward kernel runs four blocks per SM (64 registers: more gathers in flight);
// the adjoint runs two (127 registers, no spills): it takes two tiles per iteration, so
// each warp has twice the gathers in flight and needs fewer resident warps.
template <typename T, bool GRAD>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, GRAD ? 2 : 4) ecc_pair_kernel(PairArgs g) {
  __shared__ double e_warp[kWarpsPerBlock];
  __shared__ float4 recs[kWarpsPerBlock * 32 * kRec];         // anchor records, 5.5 KB per warp
  __shared__ float4 lps[GRAD ? kWarpsPerBlock * 64 : 1];      // the adjoint's tile lines, 1 KB per warp
  pair_block<T, GRAD>(g, blockIdx.x, e_warp, recs, lps);
}

// Fixed-order sum of n block partials by one block of 1024 threads: deterministic.
__device__ void reduce_fixed(const double* __restrict__ partial, int n, double* __restrict__ total, double* s) {
  double acc = 0.0;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per;
  const int end = min(n, beg + per);
  for (int i = beg; i < end; ++i) acc += partial[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s[0];
}

__global__ void __launch_bounds__(1024) reduce_kernel(const double* __restrict__ partial, int n,
                                                      double* __restrict__ total) {
  __shared__ double s[1024];
  reduce_fixed(partial, n, total, s);
}

// Serving: all active jobs' pair blocks in one persistent launch.  Each CTA takes
// the next block index from a global counter (no waiting on other CTAs), finds its
// job and runs the same per-block code as the single-scan kernel, so every job's
// partials, and its total, equal those of an evaluation of the job alone.
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 3) serve_pair_kernel(const ServeJob* __restrict__ jobs,
                                                                         const long long* __restrict__ boff,
                                                                         int n_jobs,
                                                                         unsigned long long* __restrict__ next) {
  __shared__ double e_warp[kWarpsPerBlock];
  __shared__ float4 recs[kWarpsPerBlock * 32 * kRec];  // anchor records, 5.5 KB per warp
  __shared__ float4 lps[kWarpsPerBlock * 64];          // the adjoint's tile lines, 1 KB per warp
  __shared__ long long item;
  const long long total = boff[n_jobs];
  for (;;) {
    if (threadIdx.x == 0) item = (long long)atomicAdd(next, 1ull);
    __syncthreads();
    const long long it = item;
    __syncthreads();
    if (it >= total) return;  // block-uniform
    const int j = serve_job_of(boff, n_jobs, it);
    const PairArgs g = jobs[j].pair;
    const long long blk = it - boff[j];
    switch (jobs[j].dtype) {  // block-uniform
      case 0:
        pair_block<float, true, true>(g, blk, e_warp, recs, lps);
        break;
      case 1:
        pair_block<__half, true, true>(g, blk, e_warp, recs, lps);
        break;
      default:
        pair_block<__nv_bfloat16, true, true>(g, blk, e_warp, recs, lps);
        break;
    }
  }
}

__global__ void __launch_bounds__(1024) serve_reduce_kernel(const ServeJob* __restrict__ jobs) {
  __shared__ double s[1024];
  const ServeJob& J = jobs[blockIdx.x];
  reduce_fixed(J.pair.block_partial, (int)((J.pair.n_pairs + kWarpsPerBlock - 1) / kWarpsPerBlock), J.total_out, s);
}

}  // namespace

cudaError_t launch_ecc_pairs(long long n_pairs, const PairRec* prs, const float4* ctile, int n_tiles,
                             const float4* alpha_dir, const void* sino, const float* scales, int dtype,
                             int n_alpha, int n_s, int K, int W, int H, double cauchy_c, double* per_pair,
                             int32_t* nk_out, double* block_partial, double* Gpp, int* status, int* n_blocks_out,
                             const LaunchHooks& hooks, cudaStream_t stream) {
  // The forward kernel takes two pairs per warp when that still leaves several waves of
  // blocks (the anchor pass then serves both); smaller launches keep one per warp.
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    n_sm = 1;
  const bool tiles32 = Gpp || K < kMinKappaForward64;  // the adjoint kernel (32-sample tiles)
  const bool two = !tiles32 && n_pairs >= (long long)kPairsPerForwardBlock * 4 * n_sm * kForwardWavesForTwo;
  const long long ppb = two ? kPairsPerForwardBlock : kWarpsPerBlock;
  const long long nb = (n_pairs + ppb - 1) / ppb;
  *n_blocks_out = (int)nb;
  if (nb == 0) return cudaSuccess;
  const dim3 grid((unsigned)nb), block(kWarpsPerBlock * 32);
  const float cc = (float)cauchy_c;
  const char* name = Gpp ? "ecc_pair_grad_kernel" : "ecc_pair_kernel";
  hooks.on_begin(name, stream);
  PairArgs g;
  g.n_pairs = n_pairs;
  g.prs = prs;
  g.ctile = ctile;
  g.n_tiles = n_tiles;
  g.alpha_dir = alpha_dir;
  g.sino = sino;
  g.scales = dtype == 1 ? scales : nullptr;
  pair_args_grid(g, n_alpha, n_s, W, H);
  g.K = K;
  g.cauchy_c = cc;
  g.per_pair = per_pair;
  g.nk_out = nk_out;
  g.block_partial = block_partial;
  g.Gpp = Gpp;
  g.status = status;
#define ECC_LAUNCH(TT)                                                      \
  do {                                                                      \
    if (tiles32)                                                            \
      ecc_pair_kernel<TT, true><<<grid, block, 0, stream>>>(g);             \
    else                                                                    \
      ecc_pair_kernel<TT, false><<<grid, block, 0, stream>>>(g);            \
  } while (0)
  switch (dtype) {
    case 0:
      ECC_LAUNCH(float);
      break;
    case 1:
      ECC_LAUNCH(__half);
      break;
    default:
      ECC_LAUNCH(__nv_bfloat16);
      break;
  }
#undef ECC_LAUNCH
  hooks.on_end(name, stream);
  return cudaGetLastError();
}

int serve_pairs_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, serve_pair_kernel, kWarpsPerBlock * 32, 0) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

cudaError_t launch_serve_pairs(const ServeJob* jobs, const long long* boff, int n_jobs,
                               unsigned long long* counter, int grid, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  serve_pair_kernel<<<grid, kWarpsPerBlock * 32, 0, stream>>>(jobs, boff, n_jobs, counter);
  serve_reduce_kernel<<<n_jobs, 1024, 0, stream>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partial, int n, double* total, const LaunchHooks& hooks,
                          cudaStream_t stream) {
  hooks.on_begin("reduce_kernel", stream);
  reduce_kernel<<<1, 1024, 0, stream>>>(partial, n, total);
  hooks.on_end("reduce_kernel", stream);
  return cudaGetLastError();
}

}  // namespace ecc
