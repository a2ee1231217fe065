// Pair x kappa gather-reduce of the epipolar consistency metric (Eq. 15-17).
//
// One warp owns one pair.  The pair's K sampled planes are processed in tiles of
// 32 (one plane per lane).  For every tile and view the line of the tile centre is
// an FP64 "anchor" (computed lane-parallel, one anchor per lane), split into an
// exact (alpha row, s bin) integer part and an FP32 fraction; each lane then moves
// from the anchor to its own plane with a cancellation-free FP32 formula for the
// change of (alpha, s), so that the sinogram indices carry FP64-class accuracy
// while the per-sample work stays in FP32.  Bilinear taps are gathered from the
// L2-resident sinograms, squared differences are accumulated in FP32, reduced with
// warp shuffles, normalised by N_kappa (Eq. 15), passed through the Cauchy norm
// (Eq. 16) and summed per block in a fixed order (Eq. 17, finished by the reduce
// kernel).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ecc_internal.cuh"
#include "kernels.cuh"

namespace ecc {

namespace {

constexpr int kWarpsPerBlock = 8;

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

template <typename T>
__device__ __forceinline__ float fetch(const T* __restrict__ row, int n, int n_s) {
  return (n >= 0 && n < n_s) ? Elem<T>::get(row + n) : 0.0f;
}

// Bilinear value at alpha row m (+ fraction fa toward row m+1) and s position
// n + fs of one view's sinogram.  Row n_alpha continues as row 0 at -s, negated.
template <typename T>
__device__ __forceinline__ float bilinear(const T* __restrict__ sv, int n_alpha, int n_s, int m, float fa, int n,
                                          float fs) {
  const T* r0 = sv + (size_t)m * n_s;
  const float t00 = fetch(r0, n, n_s), t01 = fetch(r0, n + 1, n_s);
  const float v0 = fmaf(fs, t01 - t00, t00);
  float v1;
  if (m + 1 < n_alpha) {
    const T* r1 = r0 + n_s;
    const float t10 = fetch(r1, n, n_s), t11 = fetch(r1, n + 1, n_s);
    v1 = fmaf(fs, t11 - t10, t10);
  } else {
    const float t10 = fetch(sv, n_s - 1 - n, n_s), t11 = fetch(sv, n_s - 2 - n, n_s);
    v1 = -fmaf(fs, t11 - t10, t10);
  }
  return fmaf(fa, v1 - v0, v0);
}

struct Anchor {
  int m0, n0;      // alpha row and s bin of the tile-centre line
  float fa0, fs0;  // fractional parts (may leave [0,1) slightly)
  float a, b;      // rate of the normal direction in the anchor frame
  float p3, s0;    // rate of the offset, anchor offset s [px]
  float sg;        // orientation fold of the anchor (+1 / -1)
};

__device__ __forceinline__ Anchor shfl_anchor(const Anchor& x, int src) {
  Anchor r;
  r.m0 = __shfl_sync(0xffffffffu, x.m0, src);
  r.n0 = __shfl_sync(0xffffffffu, x.n0, src);
  r.fa0 = __shfl_sync(0xffffffffu, x.fa0, src);
  r.fs0 = __shfl_sync(0xffffffffu, x.fs0, src);
  r.a = __shfl_sync(0xffffffffu, x.a, src);
  r.b = __shfl_sync(0xffffffffu, x.b, src);
  r.p3 = __shfl_sync(0xffffffffu, x.p3, src);
  r.s0 = __shfl_sync(0xffffffffu, x.s0, src);
  r.sg = __shfl_sync(0xffffffffu, x.sg, src);
  return r;
}

// FP64 anchor of one (view, tile): the epipolar line l = A c (centred detector
// coordinates) of the tile-centre plane, folded to alpha in [0, pi), located on
// the alpha grid against the exact row direction, and its s offset.
__device__ Anchor make_anchor(const double* __restrict__ A, double2 c, const double2* __restrict__ alpha_dir,
                              int n_alpha, float inv_dalpha, double inv_ds, double half_ns1, float inv_ds_f) {
  double l0 = A[0] * c.x + A[1] * c.y;
  double l1 = A[2] * c.x + A[3] * c.y;
  double l2 = A[4] * c.x + A[5] * c.y;
  const float cpx = (float)(-c.y), cpy = (float)c.x;  // c rotated by +90 degrees
  float q0 = (float)A[0] * cpx + (float)A[1] * cpy;
  float q1 = (float)A[2] * cpx + (float)A[3] * cpy;
  float q2 = (float)A[4] * cpx + (float)A[5] * cpy;
  Anchor r;
  r.sg = 1.0f;
  if (l1 < 0.0 || (l1 == 0.0 && l0 < 0.0)) {
    l0 = -l0; l1 = -l1; l2 = -l2;
    q0 = -q0; q1 = -q1; q2 = -q2;
    r.sg = -1.0f;
  }
  const float l0f = (float)l0, l1f = (float)l1;
  const float h = sqrtf(l0f * l0f + l1f * l1f);
  const float ih = 1.0f / h;
  const float chx = l0f * ih, chy = l1f * ih;
  r.a = (q0 * chx + q1 * chy) * ih;
  r.b = (q1 * chx - q0 * chy) * ih;
  r.p3 = q2 * ih;
  int m = (int)floorf(atan2f(l1f, l0f) * inv_dalpha);
  m = m < 0 ? 0 : (m > n_alpha - 1 ? n_alpha - 1 : m);
  const double2 u = alpha_dir[m];
  const double cr = u.x * l1 - u.y * l0;   // h sin(alpha - alpha_m), no cancellation loss in FP64
  const double dt = u.x * l0 + u.y * l1;   // h cos(alpha - alpha_m)
  const float th = atan2f((float)cr, (float)dt);
  r.m0 = m;
  r.fa0 = th * inv_dalpha;
  // s = -l2 / h = (-l2 / dt) cos(th): FP64 reciprocal from an FP32 seed and one Newton step
  double rr = (double)(1.0f / (float)dt);
  rr = fma(rr, fma(-dt, rr, 1.0), rr);
  const double sigma = -l2 * rr;
  const double is = fma(sigma, inv_ds, half_ns1);
  const double nf = floor(is);
  const float sh = sinf(0.5f * th);
  const float sigf = (float)sigma;
  r.n0 = (int)nf;
  r.fs0 = (float)(is - nf) - sigf * 2.0f * sh * sh * inv_ds_f;
  r.s0 = sigf * cosf(th);
  return r;
}

// One sample of one view: move from the anchor by delta = (lane - 15.5) dk
// (x, y: the normal direction in the anchor frame; r = |(x, y)|), fold, gather.
template <typename T>
__device__ __forceinline__ float sample(const T* __restrict__ sv, int n_alpha, int n_s, const Anchor& an, float cd,
                                        float sd, float inv_dalpha, float inv_ds_f) {
  const float x = fmaf(an.a, sd, cd);
  const float y = an.b * sd;
  const float dal = atan2f(y, x);
  const float r = sqrtf(fmaf(x, x, y * y));
  const float ab2 = fmaf(an.a, an.a, an.b * an.b);
  const float q = __fdividef(fmaf(2.0f * an.a, cd, ab2 * sd), cd + r);
  const float dls = -sd * __fdividef(fmaf(an.s0, q, an.p3), r);
  float fa = fmaf(dal, inv_dalpha, an.fa0);
  float fs = fmaf(dls, inv_ds_f, an.fs0);
  // masked samples of the other view may carry extreme offsets: clamp before the
  // integer conversion so that no index arithmetic can overflow
  const float mfl = fminf(fmaxf(floorf(fa), -4.0e6f), 4.0e6f);
  const float nfl = fminf(fmaxf(floorf(fs), -4.0e6f), 4.0e6f);
  int m = an.m0 + (int)mfl;
  int n = an.n0 + (int)nfl;
  fa -= mfl;
  fs -= nfl;
  float sign = an.sg;
  if (m >= n_alpha || m < 0) {  // alpha left [0, pi): S(alpha + pi, s) = -S(alpha, -s)
    m += m < 0 ? n_alpha : -n_alpha;
    n = n_s - 2 - n;
    fs = 1.0f - fs;
    sign = -sign;
  }
  if (m < 0 || m >= n_alpha) return 0.0f;  // only reachable for a masked sample
  return sign * bilinear(sv, n_alpha, n_s, m, fa, n, fs);
}

template <typename T>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    ecc_pair_kernel(long long n_pairs, const PairRec* __restrict__ prs, const double2* __restrict__ ctile,
                    int n_tiles, const double2* __restrict__ alpha_dir, const T* __restrict__ sino,
                    const float* __restrict__ scales, int n_alpha, int n_s, int K, double inv_ds,
                    float cauchy_c, double* __restrict__ per_pair, int32_t* __restrict__ nk_out,
                    double* __restrict__ block_partial) {
  __shared__ double e_warp[kWarpsPerBlock];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const long long p = (long long)blockIdx.x * kWarpsPerBlock + wib;
  double e_val = 0.0;
  if (p < n_pairs) {
    const PairRec& pr = prs[p];
    const int status = pr.status;
    const int nk = status == 0 ? pr.nk : 0;
    float acc = 0.0f;
    if (nk > 0) {
      const size_t vstride = (size_t)n_alpha * n_s;
      const T* sa = sino + (size_t)pr.a * vstride;
      const T* sb = sino + (size_t)pr.b * vstride;
      const float sca = scales ? scales[pr.a] : 1.0f;
      const float scb = scales ? scales[pr.b] : 1.0f;
      const float inv_dalpha = (float)((double)n_alpha / kPi);
      const double half_ns1 = 0.5 * (n_s - 1);
      const float inv_ds_f = (float)inv_ds;
      float sd, cd;
      sincosf(((float)lane - 15.5f) * (float)pr.dk, &sd, &cd);
      const int r0lo = pr.r0lo, r0hi = pr.r0hi, r1lo = pr.r1lo, r1hi = pr.r1hi;
      const double2* ct = ctile + p * n_tiles;
      for (int t0 = 0; t0 < n_tiles; t0 += 16) {
        Anchor mine;
        {
          const int v = lane >> 4;
          int t = t0 + (lane & 15);
          if (t >= n_tiles) t = n_tiles - 1;
          mine = make_anchor(pr.A[v], ct[t], alpha_dir, n_alpha, inv_dalpha, inv_ds, half_ns1, inv_ds_f);
        }
        const int tmax = min(16, n_tiles - t0);
        for (int tt = 0; tt < tmax; ++tt) {
          const Anchor aa = shfl_anchor(mine, tt);
          const Anchor ab = shfl_anchor(mine, 16 + tt);
          const int k = 32 * (t0 + tt) + lane;
          const bool valid = k < K && ((k >= r0lo && k < r0hi) || (k >= r1lo && k < r1hi));
          const float Sa = sca * sample(sa, n_alpha, n_s, aa, cd, sd, inv_dalpha, inv_ds_f);
          const float Sb = scb * sample(sb, n_alpha, n_s, ab, cd, sd, inv_dalpha, inv_ds_f);
          const float dd = Sa - Sb;
          acc += valid ? dd * dd : 0.0f;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const float d = nk > 0 ? acc / (float)nk : 0.0f;
    const float e = cauchy_c > 0.0f ? d / (1.0f + d / cauchy_c) : d;
    if (lane == 0) {
      if (per_pair) {
        per_pair[2 * p] = (double)d;
        per_pair[2 * p + 1] = (double)e;
      }
      if (nk_out) nk_out[p] = nk;
    }
    e_val = (double)e;
  }
  if (lane == 0) e_warp[wib] = e_val;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kWarpsPerBlock; ++w) s += e_warp[w];
    block_partial[blockIdx.x] = s;
  }
}

// Fixed-order sum of the block partials (one block): deterministic total.
__global__ void __launch_bounds__(1024) reduce_kernel(const double* __restrict__ partial, int n,
                                                      double* __restrict__ total) {
  __shared__ double s[1024];
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

}  // namespace

cudaError_t launch_ecc_pairs(long long n_pairs, const PairRec* prs, const double2* ctile, int n_tiles,
                             const double2* alpha_dir, const void* sino, const float* scales, int dtype,
                             int n_alpha, int n_s, int K, double inv_ds, double cauchy_c, double* per_pair,
                             int32_t* nk_out, double* block_partial, int* n_blocks_out, const LaunchHooks& hooks,
                             cudaStream_t stream) {
  const long long nb = (n_pairs + kWarpsPerBlock - 1) / kWarpsPerBlock;
  *n_blocks_out = (int)nb;
  if (nb == 0) return cudaSuccess;
  const dim3 grid((unsigned)nb), block(kWarpsPerBlock * 32);
  const float cc = (float)cauchy_c;
  hooks.on_begin("ecc_pair_kernel", stream);
  switch (dtype) {
    case 0:
      ecc_pair_kernel<float><<<grid, block, 0, stream>>>(n_pairs, prs, ctile, n_tiles, alpha_dir,
                                                         (const float*)sino, nullptr, n_alpha, n_s, K, inv_ds, cc,
                                                         per_pair, nk_out, block_partial);
      break;
    case 1:
      ecc_pair_kernel<__half><<<grid, block, 0, stream>>>(n_pairs, prs, ctile, n_tiles, alpha_dir,
                                                          (const __half*)sino, scales, n_alpha, n_s, K, inv_ds, cc,
                                                          per_pair, nk_out, block_partial);
      break;
    default:
      ecc_pair_kernel<__nv_bfloat16><<<grid, block, 0, stream>>>(n_pairs, prs, ctile, n_tiles, alpha_dir,
                                                                 (const __nv_bfloat16*)sino, nullptr, n_alpha, n_s,
                                                                 K, inv_ds, cc, per_pair, nk_out, block_partial);
      break;
  }
  hooks.on_end("ecc_pair_kernel", stream);
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
