// dRadon/ds precompute: the Grangeat intermediate function S_lambda (Eq. 1) of
// every projection on an (alpha, s) grid.
//
//   radon_table_kernel   FP64, one thread per (view, alpha row): the parameters of
//                        the detector lines (x - cx) cos a + (y - cy) sin a = sigma
//                        as 32.32 fixed-point coordinates along the interpolation
//                        axis (exact integer stepping, no FP64 in the hot loop).
//   weight_kernel        cosine pre-weight g D / sqrt(D^2 + u^2 + v^2) of each
//                        projection, stored as interpolation pairs (v[i],
//                        v[i+1] - v[i]) twice: along image rows and along image
//                        columns, each with a zero margin on both sides wide enough
//                        for the 32 lines of a warp.
//   joseph_kernel        one warp per (view, alpha, 31 consecutive s_n), a block's
//                        warps on consecutive alpha rows (shared image band): Joseph
//                        line sums (step over rows for |cos a| >= |sin a|, else over
//                        columns, linear interpolation along the other axis), one
//                        8-byte pair load and one FMA per tap.  The half-step
//                        difference in s is formed between neighbouring lanes (warp
//                        shuffle) on 8-row partial sums, so that it never cancels
//                        two large FP32 sums (Kahan-compensated across blocks); the
//                        (D^2 + s^2)/D^2 weight is applied at the end.  Lanes read
//                        consecutive pairs of one image row: coalesced, L1/L2
//                        resident.
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

// Weighted projection as interpolation pairs (v[i], v[i+1] - v[i]) along the
// interpolation axis: row-major [H][pitch_r] (pairs along x) and transposed
// [W][pitch_c] (pairs along y), the image from element pad on, zeros elsewhere
// (the pair before the image carries (0, v[0])).  A block (32, 8) covers 32x32
// pairs starting one pixel before the image; the weighted values of a 33x33 tile
// are computed once into shared memory and both planes are written coalesced.
__global__ void weight_kernel(const float* __restrict__ images, const RadonView* __restrict__ rv, int W, int H,
                              int pad, int pitch_r, int pitch_c, float2* __restrict__ wimg, size_t plane) {
  __shared__ float tile[33][34];
  const int v = blockIdx.z;
  const float* g = images + (size_t)v * W * H;
  float2* R = wimg + (size_t)v * plane;
  float2* T = R + (size_t)H * pitch_r;
  const RadonView r = rv[v];
  const int bx = (int)blockIdx.x * 32 - 1, by = (int)blockIdx.y * 32 - 1;
  for (int i = threadIdx.y * 32 + threadIdx.x; i < 33 * 33; i += 256) {
    const int ty = i / 33, tx = i % 33;
    const int x = bx + tx, y = by + ty;
    float w = 0.0f;
    if (x >= 0 && x < W && y >= 0 && y < H) {
      const float du = (float)x - r.u0, dv = (float)y - r.v0;
      w = g[(size_t)y * W + x] * (r.D / sqrtf(r.D * r.D + du * du + dv * dv));
    }
    tile[ty][tx] = w;
  }
  __syncthreads();
  for (int j = 0; j < 4; ++j) {
    const int tx = threadIdx.x, ty = threadIdx.y + 8 * j;
    const int x = bx + tx, y = by + ty;
    // pairs along x for image rows
    if (y >= 0 && y < H && x >= -1 && x < W)
      R[(size_t)y * pitch_r + x + pad] = make_float2(tile[ty][tx], tile[ty][tx + 1] - tile[ty][tx]);
    // pairs along y for image columns (threads run along y: coalesced)
    const int xo = bx + ty, yo = by + tx;
    if (xo >= 0 && xo < W && yo >= -1 && yo < H)
      T[(size_t)xo * pitch_c + yo + pad] = make_float2(tile[tx][ty], tile[tx + 1][ty] - tile[tx][ty]);
  }
}

// ---------------------------------------------------------------- Joseph line sums
//
// One warp per (view, alpha row, 31 consecutive s_n): lane i follows the line at
// the half-step offset s_{k0+i} - ds/2 (lane 31 provides the line after the last
// output).  The weighted image is stored as pairs (v[i], v[i+1] - v[i]) along the
// interpolation axis, so one tap is one 8-byte load and one FMA; lanes read
// consecutive pairs of one image row (coalesced, L1-resident).  A warp walks only
// the image rows where some of its lines meet the image (exact row range), in
// blocks of 16 rows: exact 32.32 fixed-point position at the block's first row,
// then FP32 offsets u * dy (|u| < 16, error < 2e-6 px); floor and element offset
// come from one round-down add against 1.5 * 2^23 + u * pitch.  Taps are summed
// over 8 rows, and the 8-row sum's difference to the next lane's line is added to
// a Kahan-compensated accumulator, so the half-step difference in s never cancels
// two large FP32 sums.
constexpr int kRowsPerAnchor = 16;
constexpr int kRowsPerBlock = 8;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: float ulp 1 for [2^23, 2^24)
constexpr unsigned kMagicBits = 0x4B400000u;
constexpr int kMaxPad = 160;  // wider margins: clamped variant

__device__ __forceinline__ void kahan_add(float q, float& acc, float& comp) {
  const float y = q - comp;
  const float t = acc + y;
  comp = (t - acc) - y;
  acc = t;
}

constexpr int kAlphaPerBlock = 8;  // warps per block

struct JosephArgs {
  int W, H, n_alpha, n_s;
  int pad, pitch_r, pitch_c;  // float2 elements
  size_t plane;               // float2 elements per view
  float ds;
};

// Taps of rows u in [ua, ub) of one anchor block (all 16 rows when FULL).
template <bool CLAMP, bool FULL>
__device__ __forceinline__ void joseph_block(const float2* __restrict__ rp, float f0, float dyf, float lo_c, float hi_c,
                                             const float (&Mu)[kRowsPerAnchor], int ua, int ub, float& acc,
                                             float& comp) {
#pragma unroll
  for (int i = 0; i < kRowsPerAnchor / kRowsPerBlock; ++i) {
    float s = 0.0f;
#pragma unroll
    for (int uu = 0; uu < kRowsPerBlock; ++uu) {
      const int u = i * kRowsPerBlock + uu;
      if (FULL || (u >= ua && u < ub)) {
        float xf = fmaf((float)u, dyf, f0);
        if (CLAMP) xf = fminf(fmaxf(xf, lo_c), hi_c);
        const float t = __fadd_rd(xf, Mu[u]);
        const float f = xf - (t - Mu[u]);
        const float2 vd = __ldg(rp + __float_as_uint(t));
        s += fmaf(f, vd.y, vd.x);
      }
    }
    const float nb = __shfl_down_sync(0xffffffffu, s, 1);
    kahan_add(nb - s, acc, comp);
  }
}

template <bool CLAMP>
__global__ void __launch_bounds__(32 * kAlphaPerBlock) joseph_kernel(const RadonRow* __restrict__ table,
                                                                      const RadonView* __restrict__ rv,
                                                                      const float2* __restrict__ wimg, JosephArgs g,
                                                                      float* __restrict__ out_f32,
                                                                      __nv_bfloat16* __restrict__ out_bf16) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // the warps of a block take the same 31 outputs of consecutive alpha rows: their
  // image bands largely overlap and are shared through L1
  const int v = blockIdx.z, m = (int)blockIdx.y * kAlphaPerBlock + warp;
  if (m >= g.n_alpha) return;  // warp-uniform
  const int k0 = 31 * (int)blockIdx.x;
  const int k = k0 + lane;
  const RadonRow row = table[(size_t)v * g.n_alpha + m];
  const bool rows = row.rows_mode != 0;
  const float2* img = wimg + (size_t)v * g.plane + (rows ? 0 : (size_t)g.H * g.pitch_r);
  const int pitch = rows ? g.pitch_r : g.pitch_c;
  const int n_steps = rows ? g.H : g.W;
  const int limit = rows ? g.W : g.H;
  // image rows where some lane of the warp is inside the interpolation support
  int s_lo = 0, s_hi = n_steps;
  {
    const float scale = 1.0f / 65536.0f;
    const float xa = (float)((row.B0 + (long long)k0 * row.STEP) >> 16) * scale;
    const float xb = (float)((row.B0 + (long long)(k0 + 31) * row.STEP) >> 16) * scale;
    const float dy = (float)(row.DY >> 16) * scale;
    const float mn = fminf(xa, xb) - 2.0f, mx = fmaxf(xa, xb) + 2.0f;
    const float lo_t = -1.0f, hi_t = (float)limit;
    if (fabsf(dy) > 1e-6f) {
      const float s1 = (lo_t - mx) / dy, s2 = (hi_t - mn) / dy;
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
  const float dyf = (float)((double)row.DY * (1.0 / 4294967296.0));
  const long long DY16 = (long long)kRowsPerAnchor * row.DY;
  float Mu[kRowsPerAnchor];
#pragma unroll
  for (int u = 0; u < kRowsPerAnchor; ++u) Mu[u] = kMagic + (float)(u * pitch);
  long long X = row.B0 + (long long)k * row.STEP + (long long)s_lo * row.DY;
  float acc = 0.0f, comp = 0.0f;
  // row pointers are biased by -kMagicBits elements, so that a tap's element is the
  // pointer plus the bit pattern of its round-down sum (one 32x32+64 multiply-add)
  const uint64_t img_b = reinterpret_cast<uint64_t>(img) - 8ull * kMagicBits;
  for (int j0 = s_lo; j0 < s_hi; j0 += kRowsPerAnchor) {
    const int xi0 = (int)(X >> 32);
    const float f0 = __uint_as_float(0x3f800000u | ((unsigned)X >> 9)) - 1.0f;
    const float2* rp = reinterpret_cast<const float2*>(img_b + 8ull * (uint64_t)((long long)j0 * pitch + g.pad + xi0));
    const float lo_c = (float)(-2 - xi0), hi_c = (float)(limit - xi0);
    const int n = s_hi - j0;
    if (n >= kRowsPerAnchor)
      joseph_block<CLAMP, true>(rp, f0, dyf, lo_c, hi_c, Mu, 0, n, acc, comp);
    else
      joseph_block<CLAMP, false>(rp, f0, dyf, lo_c, hi_c, Mu, 0, n, acc, comp);
    X += DY16;
  }
  if (lane < 31 && k < g.n_s) {
    const RadonView r = rv[v];
    const float sn = ((float)k - 0.5f * (float)(g.n_s - 1)) * g.ds;
    const float spp = sn - (r.u0 - 0.5f * (float)(g.W - 1)) * row.ca - (r.v0 - 0.5f * (float)(g.H - 1)) * row.sa;
    const float wgt = (r.D * r.D + spp * spp) / (r.D * r.D);
    const float val = (acc - comp) * (row.inv_len / g.ds) * wgt;
    const size_t o = ((size_t)v * g.n_alpha + m) * g.n_s + k;
    if (out_bf16)
      out_bf16[o] = __float2bfloat16_rn(val);
    else
      out_f32[o] = val;
  }
}

// FP16 storage: per-view scale = max|S| / 2^14 (1 if the view is all zero), so
// every stored value is in FP16's normal range; stored = S / scale.  The max of a view
// is split over gridDim.x blocks, each folding its part into the view's slot by an
// atomic max on the bit pattern (non-negative floats order as their bits); the slots
// start at zero and scale_finalize_kernel turns them into scales in place.
__global__ void __launch_bounds__(256) absmax_kernel(const float* __restrict__ s32, size_t per_view,
                                                     unsigned* __restrict__ max_bits) {
  const float* __restrict__ p = s32 + (size_t)blockIdx.y * per_view;
  const size_t chunk = (per_view + gridDim.x - 1) / gridDim.x;
  const size_t beg = (size_t)blockIdx.x * chunk;
  const size_t end = beg + chunk < per_view ? beg + chunk : per_view;
  float m = 0.0f;
  for (size_t i = beg + threadIdx.x; i < end; i += blockDim.x) m = fmaxf(m, fabsf(p[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(max_bits + blockIdx.y, __float_as_uint(m));
}

__global__ void scale_finalize_kernel(float* __restrict__ scales, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) scales[i] = scales[i] > 0.0f ? scales[i] / 16384.0f : 1.0f;
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
  // 1/sqrt 2 in their mode) plus the margins of the per-warp row range
  const double ds = sqrt((double)W * W + (double)H * H) / (n_s - 1);
  const int need = (int)ceil(31.0 * ds * 1.41421356237309515 + 8.0);
  return need <= kMaxPad ? need : 2;  // 2: clamped variant
}

size_t radon_plane_bytes(int W, int H, int n_s) {
  const int pad = radon_pad(W, H, n_s);
  return sizeof(float2) * ((size_t)H * (W + 2 * pad) + (size_t)W * (H + 2 * pad));
}

size_t radon_f16_stage_bytes(int n_alpha, int n_s, int batch_views) {
  return sizeof(float) * (size_t)n_alpha * n_s * batch_views;
}

cudaError_t launch_radon(const ViewRec* views, int n_views, const float* images, int W, int H, int n_alpha, int n_s,
                         int dtype, void* sino_out, float* scales_out, RadonRow* table, void* wimg,
                         float* stage, int batch_views, const LaunchHooks& hooks, cudaStream_t stream,
                         const cudaEvent_t* batch_ready) {
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
  JosephArgs jg;
  jg.W = W;
  jg.H = H;
  jg.n_alpha = n_alpha;
  jg.n_s = n_s;
  jg.pad = radon_pad(W, H, n_s);
  const bool clamp = jg.pad == 2;
  jg.pitch_r = W + 2 * jg.pad;
  jg.pitch_c = H + 2 * jg.pad;
  jg.plane = radon_plane_bytes(W, H, n_s) / sizeof(float2);
  jg.ds = (float)(sqrt((double)W * W + (double)H * H) / (n_s - 1));
  const int n_chunks = (n_s + 30) / 31;
  float2* wv = reinterpret_cast<float2*>(wimg);
  for (int v0 = 0; v0 < n_views; v0 += batch_views) {
    const int nb = min(batch_views, n_views - v0);
    cudaError_t e;
    if (v0 == 0) {  // zero margins; later batches overwrite only the pairs of the image
      e = cudaMemsetAsync(wimg, 0, sizeof(float2) * jg.plane * nb, stream);
      if (e != cudaSuccess) return e;
    }
    if (batch_ready && (e = cudaStreamWaitEvent(stream, batch_ready[v0 / batch_views], 0)) != cudaSuccess) return e;
    hooks.on_begin("weight_kernel", stream);
    weight_kernel<<<dim3((W + 32) / 32, (H + 32) / 32, nb), dim3(32, 8), 0, stream>>>(
        images + (size_t)v0 * W * H, rv + v0, W, H, jg.pad, jg.pitch_r, jg.pitch_c, wv, jg.plane);
    hooks.on_end("weight_kernel", stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const RadonRow* tb = table + (size_t)v0 * n_alpha;
    const size_t oo = (size_t)v0 * n_alpha * n_s;
    float* of = dtype == 0 ? (float*)sino_out + oo : (dtype == 1 ? stage : nullptr);
    __nv_bfloat16* ob = dtype == 2 ? (__nv_bfloat16*)sino_out + oo : nullptr;
    const dim3 grid(n_chunks, (n_alpha + kAlphaPerBlock - 1) / kAlphaPerBlock, nb), block(32 * kAlphaPerBlock);
    hooks.on_begin("joseph_kernel", stream);
    if (clamp)
      joseph_kernel<true><<<grid, block, 0, stream>>>(tb, rv + v0, wv, jg, of, ob);
    else
      joseph_kernel<false><<<grid, block, 0, stream>>>(tb, rv + v0, wv, jg, of, ob);
    hooks.on_end("joseph_kernel", stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (dtype == 1) {
      const size_t per_view = (size_t)n_alpha * n_s;
      e = cudaMemsetAsync(scales_out + v0, 0, sizeof(float) * nb, stream);
      if (e != cudaSuccess) return e;
      const unsigned per_block = 256 * 16;  // 16 elements per thread, at most 64 blocks per view
      const unsigned bpv = (unsigned)std::min<size_t>(64, (per_view + per_block - 1) / per_block);
      hooks.on_begin("absmax_kernel", stream);
      absmax_kernel<<<dim3(bpv, nb), 256, 0, stream>>>(stage, per_view, reinterpret_cast<unsigned*>(scales_out + v0));
      hooks.on_end("absmax_kernel", stream);
      scale_finalize_kernel<<<(nb + 255) / 256, 256, 0, stream>>>(scales_out + v0, nb);
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
