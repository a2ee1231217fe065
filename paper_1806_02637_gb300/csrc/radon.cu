// dRadon/ds precompute: the Grangeat intermediate function S_lambda (Eq. 1) of
// every projection on an (alpha, s) grid.
//
//   radon_table_kernel   FP64, one thread per (view, alpha row): the parameters of
//                        the detector lines (x - cx) cos a + (y - cy) sin a = sigma
//                        as 32.32 fixed-point coordinates along the interpolation
//                        axis (exact integer stepping, no FP64 in the hot loop).
//   weight_kernel        cosine pre-weight g D / sqrt(D^2 + u^2 + v^2) of each
//                        projection, written twice: row-major and transposed, each
//                        with two zero columns of padding on both sides, so that
//                        every Joseph step reads two adjacent floats of one row.
//   joseph_kernel        one warp per (view, alpha, 32 consecutive sigma): Joseph
//                        line sums (step over rows for |cos a| >= |sin a|, else over
//                        columns, linear interpolation along the other axis).  The
//                        half-step difference in s is formed tap by tap between
//                        neighbouring lanes (warp shuffle) so that it never cancels
//                        two large FP32 sums (block sums of the differences are
//                        Kahan-compensated); the (D^2 + s^2)/D^2 weight is applied
//                        at the end.  Lanes read consecutive floats of one image
//                        row: coalesced, L1/L2 resident.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ecc_internal.cuh"
#include "kernels.cuh"

namespace ecc {

namespace {

constexpr double kTwo32 = 4294967296.0;

__global__ void radon_table_kernel(const ViewRec* __restrict__ views, int n_views, int W, int H, int n_alpha,
                                   int n_s, RadonRow* __restrict__ table, RadonView* __restrict__ rv) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n_views * n_alpha) return;
  const int v = (int)(idx / n_alpha);
  const int m = (int)(idx % n_alpha);
  double sa, ca;
  sincospi((double)m / (double)n_alpha, &sa, &ca);
  const bool rows = (4 * m <= n_alpha) || (4 * m >= 3 * n_alpha);
  const double ds = sqrt((double)W * W + (double)H * H) / (n_s - 1);
  const double cx = 0.5 * (W - 1), cy = 0.5 * (H - 1);
  double B0, STEP, DY, inv_len;
  if (rows) {
    B0 = cx + (cy * sa - 0.5 * n_s * ds) / ca;
    STEP = ds / ca;
    DY = -sa / ca;
    inv_len = 1.0 / fabs(ca);
  } else {
    B0 = cy + (cx * ca - 0.5 * n_s * ds) / sa;
    STEP = ds / sa;
    DY = -ca / sa;
    inv_len = 1.0 / fabs(sa);
  }
  RadonRow r;
  r.B0 = llrint(B0 * kTwo32);
  r.STEP = llrint(STEP * kTwo32);
  r.DY = llrint(DY * kTwo32);
  r.inv_len = (float)inv_len;
  r.ca = (float)ca;
  r.sa = (float)sa;
  r.rows_mode = rows ? 1 : 0;
  table[idx] = r;
  if (m == 0) {
    const ViewRec& vr = views[v];
    RadonView o;
    o.u0 = (float)vr.u0;
    o.v0 = (float)vr.v0;
    o.D = (float)vr.D;
    o.pad = 0;
    rv[v] = o;
  }
}

// Weighted projection, row-major [H][W + 2 pad] and transposed [W][H + 2 pad]
// (data from column / row pad, zeros elsewhere).  Block (32, 8) over a 32x32 tile;
// the transpose goes through shared memory so both writes are coalesced.
__global__ void weight_kernel(const float* __restrict__ images, const RadonView* __restrict__ rv, int W, int H,
                              int pad, float* __restrict__ wimg, size_t plane) {
  __shared__ float tile[32][33];
  const int v = blockIdx.z;
  const float* g = images + (size_t)v * W * H;
  float* R = wimg + (size_t)v * plane;
  float* T = R + (size_t)H * (W + 2 * pad);
  const RadonView r = rv[v];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = 0; j < 4; ++j) {
    const int x = bx + threadIdx.x, y = by + threadIdx.y + 8 * j;
    float w = 0.0f;
    if (x < W && y < H) {
      const float du = (float)x - r.u0, dv = (float)y - r.v0;
      w = g[(size_t)y * W + x] * (r.D / sqrtf(r.D * r.D + du * du + dv * dv));
      R[(size_t)y * (W + 2 * pad) + x + pad] = w;
    }
    tile[threadIdx.y + 8 * j][threadIdx.x] = w;
  }
  __syncthreads();
  for (int j = 0; j < 4; ++j) {
    const int xo = bx + threadIdx.y + 8 * j, yo = by + threadIdx.x;
    if (xo < W && yo < H) T[(size_t)xo * (H + 2 * pad) + yo + pad] = tile[threadIdx.x][threadIdx.y + 8 * j];
  }
}

template <typename OutT>
__device__ __forceinline__ void store_out(OutT* p, float v);
template <>
__device__ __forceinline__ void store_out<float>(float* p, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_out<__half>(__half* p, float v) { *p = __float2half_rn(v); }
template <>
__device__ __forceinline__ void store_out<__nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// CLAMP = false: the zero margin (pad) is wider than the span of a warp's 32 lines
// plus the step-range margins, so every tap read stays inside the padded row
// without clamping.  CLAMP = true (coarse s grids): pad = 2 and the coordinate is
// clamped onto the zero columns.
template <typename OutT, bool CLAMP>
__global__ void __launch_bounds__(256) joseph_kernel(const RadonRow* __restrict__ table,
                                                     const RadonView* __restrict__ rv,
                                                     const float* __restrict__ wimg, size_t plane, int W, int H,
                                                     int pad, int n_alpha, int n_s, float ds, int warps_per_block,
                                                     OutT* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int v = blockIdx.z, m = blockIdx.y;
  const int chunk = blockIdx.x * warps_per_block + warp;
  const int k0 = 31 * chunk;
  if (k0 >= n_s) return;  // warp-uniform
  const int k = k0 + lane;
  const RadonRow row = table[(size_t)v * n_alpha + m];
  const bool rows = row.rows_mode != 0;
  const float* img = wimg + (size_t)v * plane + (rows ? 0 : (size_t)H * (W + 2 * pad));
  const int pitch = rows ? W + 2 * pad : H + 2 * pad;
  const int n_steps = rows ? H : W;
  const int limit = rows ? W : H;
  // steps where some lane of the warp is inside the interpolation support
  int s_lo = 0, s_hi = n_steps;
  {
    const float scale = 1.0f / 65536.0f;
    const float xa = (float)((row.B0 + (long long)k0 * row.STEP) >> 16) * scale;
    const float xb = (float)((row.B0 + (long long)(k0 + 31) * row.STEP) >> 16) * scale;
    const float dy = (float)(row.DY >> 16) * scale;
    const float mn = fminf(xa, xb) - 2.0f, mx = fmaxf(xa, xb) + 2.0f;
    const float lo_t = -1.0f, hi_t = (float)limit;
    if (fabsf(dy) > 1e-6f) {
      float s1 = (lo_t - mx) / dy, s2 = (hi_t - mn) / dy;
      // clamp in float first: nearly axis-parallel lines give huge bounds
      const float cap = (float)n_steps + 4.0f;
      const float sl = fminf(fmaxf(fminf(s1, s2), -4.0f), cap);
      const float sh = fminf(fmaxf(fmaxf(s1, s2), -4.0f), cap);
      s_lo = max(0, (int)floorf(sl) - 1);
      s_hi = min(n_steps, (int)ceilf(sh) + 2);
    } else if (mx < lo_t || mn > hi_t) {
      s_hi = 0;
    }
    if (s_hi < s_lo) s_hi = s_lo;
  }
  long long X = row.B0 + (long long)k * row.STEP + (long long)s_lo * row.DY;
  const float* base = img + (size_t)s_lo * pitch + pad;
  // Each step: tap t_j of this lane's line, t_{j+1} of the neighbour's (next sigma)
  // by shuffle, and their difference, which is small and (for neighbouring taps of
  // a smooth image) exact in FP32.  Differences are summed in 8-step blocks; the
  // block sums are added with Kahan compensation.
  float q = 0.0f, acc = 0.0f, comp = 0.0f;
  int s = s_lo;
  for (; s + 8 <= s_hi; s += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      int xi = (int)(X >> 32);
      const unsigned lo = (unsigned)(X & 0xffffffffLL);
      const float f = __uint_as_float(0x3f800000u | (lo >> 9)) - 1.0f;
      if (CLAMP) xi = min(max(xi, -2), limit);
      const float* rp = base + xi;
      const float v0 = __ldg(rp), v1 = __ldg(rp + 1);
      const float t = fmaf(f, v1 - v0, v0);
      const float nb = __shfl_down_sync(0xffffffffu, t, 1);
      q += nb - t;
      X += row.DY;
      base += pitch;
    }
    const float y = q - comp;
    const float tt = acc + y;
    comp = (tt - acc) - y;
    acc = tt;
    q = 0.0f;
  }
  for (; s < s_hi; ++s) {
    int xi = (int)(X >> 32);
    const unsigned lo = (unsigned)(X & 0xffffffffLL);
    const float f = __uint_as_float(0x3f800000u | (lo >> 9)) - 1.0f;
    if (CLAMP) xi = min(max(xi, -2), limit);
    const float* rp = base + xi;
    const float v0 = __ldg(rp), v1 = __ldg(rp + 1);
    const float t = fmaf(f, v1 - v0, v0);
    const float nb = __shfl_down_sync(0xffffffffu, t, 1);
    q += nb - t;
    X += row.DY;
    base += pitch;
  }
  {
    const float y = q - comp;
    acc = acc + y;
  }
  if (lane < 31 && k < n_s) {
    const RadonView r = rv[v];
    const float sn = ((float)k - 0.5f * (float)(n_s - 1)) * ds;
    const float spp = sn - (r.u0 - 0.5f * (float)(W - 1)) * row.ca - (r.v0 - 0.5f * (float)(H - 1)) * row.sa;
    const float wgt = (r.D * r.D + spp * spp) / (r.D * r.D);
    store_out<OutT>(out + ((size_t)v * n_alpha + m) * n_s + k, acc * (row.inv_len / ds) * wgt);
  }
}

// FP16 storage: per-view scale = max|S| / 2^14 (1 if the view is all zero), so
// every stored value is in FP16's normal range; stored = S / scale.
__global__ void __launch_bounds__(256) absmax_scale_kernel(const float* __restrict__ s32, size_t per_view,
                                                          float* __restrict__ scales) {
  __shared__ float sh[256];
  const float* p = s32 + (size_t)blockIdx.x * per_view;
  float m = 0.0f;
  for (size_t i = threadIdx.x; i < per_view; i += blockDim.x) m = fmaxf(m, fabsf(p[i]));
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) scales[blockIdx.x] = sh[0] > 0.0f ? sh[0] / 16384.0f : 1.0f;
}

__global__ void quantize_f16_kernel(const float* __restrict__ s32, size_t per_view, size_t n,
                                    const float* __restrict__ scales, __half* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = __float2half_rn(s32[i] / scales[i / per_view]);
}

}  // namespace

int radon_pad(int W, int H, int n_s) {
  // span of 32 neighbouring lines along the interpolation axis (|cos| or |sin| >=
  // 1/sqrt 2 in their mode) plus the margins of the per-warp step range
  const double ds = sqrt((double)W * W + (double)H * H) / (n_s - 1);
  const int need = (int)ceil(31.0 * ds * 1.41421356237309515 + 8.0);
  const int pad = (need + 3) / 4 * 4;
  return pad <= 160 ? pad : 2;  // 2: clamped variant
}

size_t radon_plane_floats(int W, int H, int n_s) {
  const int pad = radon_pad(W, H, n_s);
  return (size_t)H * (W + 2 * pad) + (size_t)W * (H + 2 * pad);
}

size_t radon_f16_stage_bytes(int n_alpha, int n_s, int batch_views) {
  return sizeof(float) * (size_t)n_alpha * n_s * batch_views;
}

cudaError_t launch_radon(const ViewRec* views, int n_views, const float* images, int W, int H, int n_alpha, int n_s,
                         int dtype, void* sino_out, float* scales_out, RadonRow* table, float* wimg,
                         float* stage, int batch_views, const LaunchHooks& hooks, cudaStream_t stream) {
  // table and per-view weights (RadonView array sits right after the table)
  RadonView* rv = reinterpret_cast<RadonView*>(table + (size_t)n_views * n_alpha);
  {
    const long long n = (long long)n_views * n_alpha;
    hooks.on_begin("radon_table_kernel", stream);
    radon_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(views, n_views, W, H, n_alpha, n_s, table,
                                                                       rv);
    hooks.on_end("radon_table_kernel", stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int pad = radon_pad(W, H, n_s);
  const bool clamp = pad == 2;
  const size_t plane = radon_plane_floats(W, H, n_s);
  const float ds = (float)(sqrt((double)W * W + (double)H * H) / (n_s - 1));
  const int n_chunks = (n_s + 30) / 31;
  const int blocks_x = (n_chunks + 7) / 8;
  const int wpb = (n_chunks + blocks_x - 1) / blocks_x;
  for (int v0 = 0; v0 < n_views; v0 += batch_views) {
    const int nb = min(batch_views, n_views - v0);
    cudaError_t e = cudaMemsetAsync(wimg, 0, sizeof(float) * plane * nb, stream);
    if (e != cudaSuccess) return e;
    hooks.on_begin("weight_kernel", stream);
    weight_kernel<<<dim3((W + 31) / 32, (H + 31) / 32, nb), dim3(32, 8), 0, stream>>>(
        images + (size_t)v0 * W * H, rv + v0, W, H, pad, wimg, plane);
    hooks.on_end("weight_kernel", stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid(blocks_x, n_alpha, nb), block(32 * wpb);
    const RadonRow* tb = table + (size_t)v0 * n_alpha;
    hooks.on_begin("joseph_kernel", stream);
#define JOSEPH(OT, OUTPTR)                                                                                    \
  do {                                                                                                      \
    if (clamp)                                                                                              \
      joseph_kernel<OT, true><<<grid, block, 0, stream>>>(tb, rv + v0, wimg, plane, W, H, pad, n_alpha, n_s, \
                                                          ds, wpb, OUTPTR);                                   \
    else                                                                                                    \
      joseph_kernel<OT, false><<<grid, block, 0, stream>>>(tb, rv + v0, wimg, plane, W, H, pad, n_alpha, n_s, \
                                                           ds, wpb, OUTPTR);                                  \
  } while (0)
    switch (dtype) {
      case 0:
        JOSEPH(float, (float*)sino_out + (size_t)v0 * n_alpha * n_s);
        break;
      case 1:  // FP32 into the staging buffer; scaled and rounded to FP16 below
        JOSEPH(float, stage);
        break;
      default:
        JOSEPH(__nv_bfloat16, (__nv_bfloat16*)sino_out + (size_t)v0 * n_alpha * n_s);
        break;
    }
#undef JOSEPH
    hooks.on_end("joseph_kernel", stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (dtype == 1) {
      const size_t per_view = (size_t)n_alpha * n_s;
      hooks.on_begin("absmax_scale_kernel", stream);
      absmax_scale_kernel<<<nb, 256, 0, stream>>>(stage, per_view, scales_out + v0);
      hooks.on_end("absmax_scale_kernel", stream);
      const size_t n = per_view * nb;
      hooks.on_begin("quantize_f16_kernel", stream);
      quantize_f16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(
          stage, per_view, n, scales_out + v0, (__half*)sino_out + (size_t)v0 * per_view);
      hooks.on_end("quantize_f16_kernel", stream);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace ecc
