// C ABI of the ECC library: context, argument validation, scratch memory and the
// launch sequence of each entry point.  See include/ecc.h for the contract.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ecc.h"
#include "ecc_internal.cuh"
#include "kernels.cuh"
#include "serve.h"

namespace {

struct Buf {
  void* p = nullptr;
  size_t n = 0;
};

thread_local std::string g_create_error;

}  // namespace

struct ProfRec {
  const char* name;
  cudaEvent_t b, e;
};

struct ecc_ctx {
  long long launches = 0;
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  int device = 0;
  size_t budget = 0;
  size_t held = 0;
  std::string err;
  int* d_status = nullptr;
  Buf views, pairs, ctile, adir, perpair, nk, partial, rtable, wimg, stage;
  Buf vtan, Gpp, gq;  // adjoint scratch: view tangents (theta), d e / d A, d e / d (C, up, cofc)
  Buf vtanP;          // view tangents with respect to P
  // the alpha-row direction table in adir was written for adir_n rows at adir_ptr
  // (calls on one context share one stream, so a later call finds it complete)
  int adir_n = 0;
  const void* adir_ptr = nullptr;
  // sampling of the last evaluation (for ecc_evaluate_frozen)
  bool samp_valid = false;
  int samp_views = 0, samp_pairs = 0, samp_K = 0, samp_W = 0, samp_H = 0;
  const void* samp_pair_ptr = nullptr;
  Buf h_P, h_img, h_sino, h_total;  // buffers of the host-buffer entry point
  cudaStream_t copy_stream = nullptr;  // its image uploads, per precompute batch
  ecc_serve* serve = nullptr;       // serving scheduler, created by the first ecc_submit
};

namespace {

int fail(ecc_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return code;
}

int cuda_fail(ecc_ctx* c, cudaError_t e, const char* what) {
  return fail(c, ECC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Grow-only scratch allocation, bounded by the context budget.
int ensure(ecc_ctx* c, Buf& b, size_t bytes, const char* name) {
  if (bytes == 0) bytes = 16;
  if (b.n >= bytes) return ECC_OK;
  const size_t old = b.n;
  if (c->budget && c->held - old + bytes > c->budget)
    return fail(c, ECC_ENOMEM, "scratch '%s' of %zu bytes exceeds the context budget (%zu held of %zu)", name, bytes,
                c->held, c->budget);
  if (b.p) {
    cudaFree(b.p);  // synchronises the device: no kernel still uses the old buffer
    b.p = nullptr;
    b.n = 0;
    c->held -= old;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(c, ECC_ENOMEM, "cudaMalloc of scratch '%s' (%zu bytes): %s", name, bytes, cudaGetErrorString(e));
  }
  b.n = bytes;
  c->held += bytes;
  return ECC_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

cudaEvent_t pooled_event(ecc_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void hook_begin(void* vc, const char* name, cudaStream_t s) {
  ecc_ctx* c = (ecc_ctx*)vc;
  ++c->launches;
  if (!c->prof) return;
  cudaEvent_t b = pooled_event(c);
  if (b) cudaEventRecord(b, s);
  c->recs.push_back({name, b, nullptr});
}

void hook_end(void* vc, const char* name, cudaStream_t s) {
  ecc_ctx* c = (ecc_ctx*)vc;
  (void)name;
  if (!c->prof || c->recs.empty()) return;
  cudaEvent_t e = pooled_event(c);
  if (e) cudaEventRecord(e, s);
  c->recs.back().e = e;
}

ecc::LaunchHooks hooks_of(ecc_ctx* c) {
  ecc::LaunchHooks h;
  h.begin = hook_begin;
  h.end = hook_end;
  h.ctx = c;
  return h;
}

int check_geometry_args(ecc_ctx* c, int n_views, const void* P, int W, int H, int n_alpha, int n_s, int dtype) {
  if (n_views < 1) return fail(c, ECC_EINVAL, "n_views must be >= 1 (got %d)", n_views);
  if (!P) return fail(c, ECC_EINVAL, "P is NULL");
  if (W < 2 || H < 2 || W > 16384 || H > 16384) return fail(c, ECC_EINVAL, "detector %dx%d out of range", W, H);
  if (n_alpha < 4 || n_alpha > 65535) return fail(c, ECC_EINVAL, "n_alpha %d out of range [4, 65535]", n_alpha);
  if (n_s < 2 || n_s > 65535) return fail(c, ECC_EINVAL, "n_s %d out of range [2, 65535]", n_s);
  if (dtype != ECC_F32 && dtype != ECC_F16 && dtype != ECC_BF16) return fail(c, ECC_EINVAL, "unknown dtype %d", dtype);
  return ECC_OK;
}


// Views per dRadon/ds batch: the weighted images of a batch take at most 256 MiB.
int radon_batch_views(int n_views, int W, int H, int n_s) {
  const size_t plane = ecc::radon_plane_bytes(W, H, n_s);
  const size_t max_batch_bytes = (size_t)256 << 20;
  return (int)std::max<size_t>(1, std::min<size_t>((size_t)n_views, max_batch_bytes / plane));
}

// batch_ready (or NULL): one event per batch, which the stream waits for before the
// batch reads its images.
int run_precompute(ecc_ctx* c, int n_views, const double* P, const float* images, int W, int H, int n_alpha, int n_s,
                   int dtype, void* sino_out, float* scales_out, cudaStream_t s,
                   const cudaEvent_t* batch_ready = nullptr) {
  int rc;
  if ((rc = ensure(c, c->views, sizeof(ecc::ViewRec) * (size_t)n_views, "views")) != ECC_OK) return rc;
  const size_t tbytes = sizeof(ecc::RadonRow) * (size_t)n_views * n_alpha + sizeof(ecc::RadonView) * (size_t)n_views;
  if ((rc = ensure(c, c->rtable, tbytes, "radon table")) != ECC_OK) return rc;
  const size_t plane = ecc::radon_plane_bytes(W, H, n_s);
  const int batch = radon_batch_views(n_views, W, H, n_s);
  if ((rc = ensure(c, c->wimg, plane * (size_t)batch, "weighted images")) != ECC_OK) return rc;
  if (dtype == ECC_F16 &&
      (rc = ensure(c, c->stage, ecc::radon_f16_stage_bytes(n_alpha, n_s, batch), "FP16 staging")) != ECC_OK)
    return rc;
  const ecc::LaunchHooks hk = hooks_of(c);
  hk.on_begin("view_setup_kernel", s);
  ecc::view_setup_kernel<<<(n_views + 127) / 128, 128, 0, s>>>(n_views, P, nullptr, W, H, (ecc::ViewRec*)c->views.p,
                                                              c->d_status);
  hk.on_end("view_setup_kernel", s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "view set-up launch");
  e = ecc::launch_radon((const ecc::ViewRec*)c->views.p, n_views, images, W, H, n_alpha, n_s, dtype, sino_out,
                        scales_out, (ecc::RadonRow*)c->rtable.p, c->wimg.p, (float*)c->stage.p, batch, hk, s,
                        batch_ready);
  if (e != cudaSuccess) return cuda_fail(c, e, "radon launch");
  return ECC_OK;
}

int run_evaluate(ecc_ctx* c, int n_views, const double* P, const double* motion, const void* sino,
                 const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa, double cauchy_c,
                 const int32_t* pairs, int n_pairs, double* total, double* per_pair, int32_t* nkappa, double* grad,
                 double* grad_P, bool reuse, cudaStream_t s) {
  int rc;
  cudaError_t e;
  if (reuse && !(c->samp_valid && c->samp_views == n_views && c->samp_pairs == n_pairs && c->samp_K == n_kappa &&
                 c->samp_W == W && c->samp_H == H && c->samp_pair_ptr == (const void*)pairs))
    return fail(c, ECC_EINVAL, "no previous evaluation on this context with the same views, pairs and n_kappa");
  if (grad && n_pairs == 0) {
    e = cudaMemsetAsync(grad, 0, sizeof(double) * 6 * (size_t)n_views, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset grad");
  }
  if (grad_P && n_pairs == 0) {
    e = cudaMemsetAsync(grad_P, 0, sizeof(double) * 12 * (size_t)n_views, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset grad_P");
  }
  if (n_pairs == 0) {
    e = cudaMemsetAsync(total, 0, sizeof(double), s);
    return e == cudaSuccess ? ECC_OK : cuda_fail(c, e, "memset total");
  }
  const int n_tiles = (n_kappa + 31) / 32;
  const long long np = n_pairs;
  const long long n_blocks = (np + 7) / 8;
  if ((rc = ensure(c, c->views, sizeof(ecc::ViewRec) * (size_t)n_views, "views")) != ECC_OK) return rc;
  if ((rc = ensure(c, c->pairs, sizeof(ecc::PairRec) * (size_t)np, "pairs")) != ECC_OK) return rc;
  if ((rc = ensure(c, c->ctile, sizeof(float4) * (size_t)np * n_tiles, "tile directions")) != ECC_OK) return rc;
  if ((rc = ensure(c, c->adir, sizeof(float4) * (size_t)n_alpha, "alpha directions")) != ECC_OK) return rc;
  if ((rc = ensure(c, c->partial, sizeof(double) * (size_t)n_blocks, "block partials")) != ECC_OK) return rc;
  if (!per_pair) {
    if ((rc = ensure(c, c->perpair, sizeof(double) * 2 * (size_t)np, "per-pair")) != ECC_OK) return rc;
    per_pair = (double*)c->perpair.p;
  }
  if (grad || grad_P) {
    if ((rc = ensure(c, c->Gpp, sizeof(double) * 12 * (size_t)np, "pair adjoints")) != ECC_OK) return rc;
  }
  if (grad || grad_P) {
    if ((rc = ensure(c, c->gq, sizeof(float2) * 30 * (size_t)np, "pair q gradients")) != ECC_OK) return rc;
  }
  if (grad) {
    if ((rc = ensure(c, c->vtan, sizeof(ecc::ViewTan) * (size_t)n_views, "view tangents")) != ECC_OK) return rc;
  }
  if (grad_P) {
    if ((rc = ensure(c, c->vtanP, sizeof(ecc::ViewTanP) * (size_t)n_views, "view P tangents")) != ECC_OK) return rc;
  }
  if (!reuse) c->samp_valid = false;
  const ecc::LaunchHooks hk = hooks_of(c);
  hk.on_begin("view_setup_kernel", s);
  ecc::view_setup_kernel<<<(n_views + 127) / 128, 128, 0, s>>>(n_views, P, motion, W, H, (ecc::ViewRec*)c->views.p,
                                                              c->d_status);
  hk.on_end("view_setup_kernel", s);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "view set-up launch");
  if (c->adir_n != n_alpha || c->adir_ptr != c->adir.p) {  // the table depends on n_alpha only
    hk.on_begin("alpha_dir_kernel", s);
    ecc::alpha_dir_kernel<<<(n_alpha + 255) / 256, 256, 0, s>>>(n_alpha, (float4*)c->adir.p);
    hk.on_end("alpha_dir_kernel", s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "alpha table launch");
    c->adir_n = n_alpha;
    c->adir_ptr = c->adir.p;
  }
  // One pair set-up launch, then one pair-kernel launch, on the caller's stream.  (Set-up
  // chunks on a second stream beside the pair kernel's chunks were measured slower: the
  // two kernels sharing SMs slowed each other, 0.707 -> 0.765 ms on the 496-view scan.)
  hk.on_begin("pair_setup_kernel", s);
  ecc::pair_setup_kernel<<<(unsigned)((np + 127) / 128), 128, 0, s>>>(
      n_views, 0, np, pairs, (const ecc::ViewRec*)c->views.p, W, H, n_kappa, (ecc::PairRec*)c->pairs.p,
      (float4*)c->ctile.p, n_tiles, reuse ? 1 : 0, c->d_status);
  hk.on_end("pair_setup_kernel", s);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "pair set-up launch");
  int nb = 0;
  e = ecc::launch_ecc_pairs(np, (const ecc::PairRec*)c->pairs.p, (const float4*)c->ctile.p, n_tiles,
                            (const float4*)c->adir.p, sino, scales, dtype, n_alpha, n_s, n_kappa, W, H, cauchy_c,
                            per_pair, nkappa, (double*)c->partial.p, (grad || grad_P) ? (double*)c->Gpp.p : nullptr,
                            c->d_status, &nb, hk, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pair kernel launch");
  e = ecc::launch_reduce((const double*)c->partial.p, nb, total, hk, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "reduce launch");
  if (grad || grad_P) {
    // d e / d (C, up, cofc) per pair, shared by both gradients
    hk.on_begin("pair_grad_q_kernel", s);
    ecc::pair_grad_q_kernel<<<(unsigned)((np + 63) / 64), 64, 0, s>>>(np, (const ecc::PairRec*)c->pairs.p,
                                                                      (const ecc::ViewRec*)c->views.p,
                                                                      (const double*)c->Gpp.p, (float2*)c->gq.p);
    hk.on_end("pair_grad_q_kernel", s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "pair q gradient launch");
  }
  if (grad) {
    hk.on_begin("view_tangent_kernel", s);
    ecc::view_tangent_kernel<<<(6 * n_views + 95) / 96, 96, 0, s>>>(n_views, P, motion, W, H,
                                                                   (ecc::ViewTan*)c->vtan.p);
    hk.on_end("view_tangent_kernel", s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "view tangent launch");
    hk.on_begin("view_grad_theta_kernel", s);
    ecc::view_grad_theta_kernel<<<n_views, 256, 0, s>>>(n_views, np, pairs, (const float2*)c->gq.p,
                                                        (const ecc::ViewTan*)c->vtan.p, grad);
    hk.on_end("view_grad_theta_kernel", s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "gradient reduce launch");
  }
  if (grad_P) {
    hk.on_begin("view_tangent_P_kernel", s);
    ecc::view_tangent_P_kernel<<<(12 * n_views + 95) / 96, 96, 0, s>>>(n_views, P, motion, W, H,
                                                                       (ecc::ViewTanP*)c->vtanP.p);
    hk.on_end("view_tangent_P_kernel", s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "view P tangent launch");
    hk.on_begin("view_grad_P_kernel", s);
    ecc::view_grad_P_kernel<<<n_views, 256, 0, s>>>(n_views, np, pairs, (const float2*)c->gq.p,
                                                    (const ecc::ViewTanP*)c->vtanP.p, grad_P);
    hk.on_end("view_grad_P_kernel", s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "P gradient reduce launch");
  }
  if (!reuse) {
    c->samp_valid = true;
    c->samp_views = n_views;
    c->samp_pairs = n_pairs;
    c->samp_K = n_kappa;
    c->samp_W = W;
    c->samp_H = H;
    c->samp_pair_ptr = pairs;
  }
  return ECC_OK;
}

}  // namespace

extern "C" {

int ecc_version(void) { return 100; }

int ecc_create(ecc_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return fail(nullptr, ECC_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, ECC_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  }
  if (device < 0 || device >= n) return fail(nullptr, ECC_EINVAL, "device %d out of range (%d devices)", device, n);
  DeviceGuard g(device);
  ecc_ctx* c = new ecc_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes;
  e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(nullptr, ECC_ECUDA, "context allocation: %s", cudaGetErrorString(e));
  }
  *out = c;
  return ECC_OK;
}

void ecc_destroy(ecc_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  ecc::serve_destroy(c->serve);
  cudaDeviceSynchronize();
  Buf* bufs[] = {&c->views, &c->pairs, &c->ctile, &c->adir, &c->perpair, &c->nk, &c->partial, &c->rtable, &c->wimg,
                 &c->vtan, &c->Gpp, &c->gq, &c->vtanP, &c->stage, &c->h_P, &c->h_img, &c->h_sino, &c->h_total};
  for (Buf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->d_status) cudaFree(c->d_status);
  for (const ProfRec& r : c->recs) {
    if (r.b) cudaEventDestroy(r.b);
    if (r.e) cudaEventDestroy(r.e);
  }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  delete c;
}

const char* ecc_last_error(const ecc_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int ecc_status(ecc_ctx* c, void* stream, int* flags) {
  if (!c || !flags) return fail(c, ECC_EINVAL, "ctx or flags is NULL");
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "status read");
  *flags = h;
  return ECC_OK;
}

long long ecc_kernel_launches(const ecc_ctx* c) { return c ? c->launches : -1; }

int ecc_profile_enable(ecc_ctx* c, int enable) {
  if (!c) return fail(nullptr, ECC_EINVAL, "ctx is NULL");
  c->prof = enable != 0;
  return ECC_OK;
}

int ecc_profile_read(ecc_ctx* c, void* stream, int max_entries, char* names, long long* launches,
                     double* total_ms, int* n_entries) {
  if (!c || !n_entries || max_entries < 0 || (max_entries > 0 && (!names || !launches || !total_ms)))
    return fail(c, ECC_EINVAL, "invalid profile_read arguments");
  DeviceGuard g(c->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile stream sync");
  std::vector<std::string> nm;
  std::vector<long long> cnt;
  std::vector<double> ms;
  for (const ProfRec& r : c->recs) {
    float t = 0.0f;
    if (r.b && r.e && cudaEventElapsedTime(&t, r.b, r.e) != cudaSuccess) {
      cudaGetLastError();
      t = 0.0f;
    }
    size_t k = 0;
    while (k < nm.size() && nm[k] != r.name) ++k;
    if (k == nm.size()) {
      nm.push_back(r.name);
      cnt.push_back(0);
      ms.push_back(0.0);
    }
    cnt[k] += 1;
    ms[k] += t;
    if (r.b) c->pool.push_back(r.b);
    if (r.e) c->pool.push_back(r.e);
  }
  c->recs.clear();
  const int n = (int)std::min<size_t>(nm.size(), (size_t)max_entries);
  for (int k = 0; k < n; ++k) {
    std::snprintf(names + 32 * k, 32, "%s", nm[k].c_str());
    launches[k] = cnt[k];
    total_ms[k] = ms[k];
  }
  *n_entries = n;
  return ECC_OK;
}

int ecc_precompute_radon_derivative(ecc_ctx* c, int n_views, const double* P, const float* images, int W, int H,
                                    int n_alpha, int n_s, int dtype, void* sino_out, float* scales_out,
                                    void* stream) {
  if (!c) return fail(nullptr, ECC_EINVAL, "ctx is NULL");
  int rc = check_geometry_args(c, n_views, P, W, H, n_alpha, n_s, dtype);
  if (rc != ECC_OK) return rc;
  if (!images || !sino_out) return fail(c, ECC_EINVAL, "images or sino_out is NULL");
  if (dtype == ECC_F16 && !scales_out) return fail(c, ECC_EINVAL, "ECC_F16 needs scales_out");
  DeviceGuard g(c->device);
  return run_precompute(c, n_views, P, images, W, H, n_alpha, n_s, dtype, sino_out, scales_out,
                        (cudaStream_t)stream);
}

namespace {
int check_eval_args(ecc_ctx* c, int n_views, const double* P, const void* sino, const float* scales, int W, int H,
                    int n_alpha, int n_s, int dtype, int n_kappa, double cauchy_c, const int32_t* pairs, int n_pairs,
                    const double* total) {
  if (!c) return fail(nullptr, ECC_EINVAL, "ctx is NULL");
  int rc = check_geometry_args(c, n_views, P, W, H, n_alpha, n_s, dtype);
  if (rc != ECC_OK) return rc;
  if (!sino || !total) return fail(c, ECC_EINVAL, "sino or total is NULL");
  if (dtype == ECC_F16 && !scales) return fail(c, ECC_EINVAL, "ECC_F16 needs scales");
  if (n_kappa < 1 || n_kappa > 65536) return fail(c, ECC_EINVAL, "n_kappa %d out of range [1, 65536]", n_kappa);
  if (n_pairs < 0) return fail(c, ECC_EINVAL, "n_pairs %d < 0", n_pairs);
  if (!pairs && n_pairs > 0) {
    const long long all = (long long)n_views * (n_views - 1) / 2;
    if (all != n_pairs)
      return fail(c, ECC_EINVAL, "pairs is NULL but n_pairs (%d) != n_views (n_views - 1) / 2 (%lld)", n_pairs, all);
  }
  if (!std::isfinite(cauchy_c)) return fail(c, ECC_EINVAL, "cauchy_c is not finite");
  return ECC_OK;
}
}  // namespace

int ecc_evaluate(ecc_ctx* c, int n_views, const double* P, const double* motion, const void* sino,
                 const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa, double cauchy_c,
                 const int32_t* pairs, int n_pairs, double* total, double* per_pair, int32_t* nkappa, void* stream) {
  int rc = check_eval_args(c, n_views, P, sino, scales, W, H, n_alpha, n_s, dtype, n_kappa, cauchy_c, pairs, n_pairs,
                           total);
  if (rc != ECC_OK) return rc;
  DeviceGuard g(c->device);
  return run_evaluate(c, n_views, P, motion, sino, scales, W, H, n_alpha, n_s, dtype, n_kappa, cauchy_c, pairs,
                      n_pairs, total, per_pair, nkappa, nullptr, nullptr, false, (cudaStream_t)stream);
}

int ecc_evaluate_frozen(ecc_ctx* c, int n_views, const double* P, const double* motion, const void* sino,
                        const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa,
                        double cauchy_c, const int32_t* pairs, int n_pairs, double* total, double* per_pair,
                        int32_t* nkappa, void* stream) {
  int rc = check_eval_args(c, n_views, P, sino, scales, W, H, n_alpha, n_s, dtype, n_kappa, cauchy_c, pairs, n_pairs,
                           total);
  if (rc != ECC_OK) return rc;
  DeviceGuard g(c->device);
  return run_evaluate(c, n_views, P, motion, sino, scales, W, H, n_alpha, n_s, dtype, n_kappa, cauchy_c, pairs,
                      n_pairs, total, per_pair, nkappa, nullptr, nullptr, true, (cudaStream_t)stream);
}

int ecc_evaluate_grad(ecc_ctx* c, int n_views, const double* P, const double* motion, const void* sino,
                      const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa,
                      double cauchy_c, const int32_t* pairs, int n_pairs, double* total, double* per_pair,
                      int32_t* nkappa, double* grad, void* stream) {
  int rc = check_eval_args(c, n_views, P, sino, scales, W, H, n_alpha, n_s, dtype, n_kappa, cauchy_c, pairs, n_pairs,
                           total);
  if (rc != ECC_OK) return rc;
  if (!grad) return fail(c, ECC_EINVAL, "grad is NULL");
  DeviceGuard g(c->device);
  return run_evaluate(c, n_views, P, motion, sino, scales, W, H, n_alpha, n_s, dtype, n_kappa, cauchy_c, pairs,
                      n_pairs, total, per_pair, nkappa, grad, nullptr, false, (cudaStream_t)stream);
}

int ecc_evaluate_grad_projection(ecc_ctx* c, int n_views, const double* P, const double* motion, const void* sino,
                                 const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa,
                                 double cauchy_c, const int32_t* pairs, int n_pairs, double* total,
                                 double* per_pair, int32_t* nkappa, double* grad_P, void* stream) {
  int rc = check_eval_args(c, n_views, P, sino, scales, W, H, n_alpha, n_s, dtype, n_kappa, cauchy_c, pairs, n_pairs,
                           total);
  if (rc != ECC_OK) return rc;
  if (!grad_P) return fail(c, ECC_EINVAL, "grad_P is NULL");
  DeviceGuard g(c->device);
  return run_evaluate(c, n_views, P, motion, sino, scales, W, H, n_alpha, n_s, dtype, n_kappa, cauchy_c, pairs,
                      n_pairs, total, per_pair, nkappa, nullptr, grad_P, false, (cudaStream_t)stream);
}

int ecc_scan_consistency_host(ecc_ctx* c, int n_views, const double* P_host, const float* images_host, int W,
                              int H, int n_alpha, int n_s, int n_kappa, double cauchy_c, double* total_host,
                              void* stream) {
  if (!c) return fail(nullptr, ECC_EINVAL, "ctx is NULL");
  int rc = check_geometry_args(c, n_views, P_host, W, H, n_alpha, n_s, ECC_F32);
  if (rc != ECC_OK) return rc;
  if (!images_host || !total_host) return fail(c, ECC_EINVAL, "images_host or total_host is NULL");
  if (n_views < 2) return fail(c, ECC_EINVAL, "need at least two views");
  if (n_kappa < 1 || n_kappa > 65536) return fail(c, ECC_EINVAL, "n_kappa %d out of range [1, 65536]", n_kappa);
  const long long np = (long long)n_views * (n_views - 1) / 2;
  if (np > 0x7fffffffLL) return fail(c, ECC_EINVAL, "too many pairs");
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t pb = sizeof(double) * 12 * (size_t)n_views;
  const size_t ib = sizeof(float) * (size_t)W * H * n_views;
  const size_t sb = sizeof(float) * (size_t)n_alpha * n_s * n_views;
  if ((rc = ensure(c, c->h_P, pb, "host-call P")) != ECC_OK) return rc;
  if ((rc = ensure(c, c->h_img, ib, "host-call images")) != ECC_OK) return rc;
  if ((rc = ensure(c, c->h_sino, sb, "host-call sinograms")) != ECC_OK) return rc;
  if ((rc = ensure(c, c->h_total, sizeof(double), "host-call total")) != ECC_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(c->h_P.p, P_host, pb, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  // From pinned host memory the images go up per precompute batch on a second stream,
  // so that the upload of batch b + 1 overlaps the projection of batch b; pageable
  // memory (whose asynchronous copies block the host) is copied in one piece.
  const int batch = radon_batch_views(n_views, W, H, n_s);
  const int n_batches = (n_views + batch - 1) / batch;
  cudaPointerAttributes pa;
  const bool pinned = cudaPointerGetAttributes(&pa, images_host) == cudaSuccess && pa.type == cudaMemoryTypeHost;
  (void)cudaGetLastError();  // a pageable pointer may leave an error from the query
  struct Events {
    std::vector<cudaEvent_t> ev;
    ~Events() {
      for (cudaEvent_t x : ev) cudaEventDestroy(x);
    }
  } ready;
  if (pinned && n_batches > 1) {
    if (!c->copy_stream && (e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(c, e, "copy stream");
    for (int b = 0; b <= n_batches && e == cudaSuccess; ++b) {  // [n_batches]: the start marker
      cudaEvent_t x;
      e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
      if (e == cudaSuccess) ready.ev.push_back(x);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "upload events");
    // the uploads follow all earlier work of the stream (earlier calls read these buffers)
    e = cudaEventRecord(ready.ev[n_batches], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, ready.ev[n_batches], 0);
    for (int b = 0; b < n_batches && e == cudaSuccess; ++b) {
      const size_t v0 = (size_t)b * batch, nv = (size_t)std::min(batch, n_views - b * batch);
      const size_t px = (size_t)W * H;
      e = cudaMemcpyAsync((float*)c->h_img.p + v0 * px, images_host + v0 * px, sizeof(float) * px * nv,
                          cudaMemcpyHostToDevice, c->copy_stream);
      if (e == cudaSuccess) e = cudaEventRecord(ready.ev[b], c->copy_stream);
    }
  } else {
    e = cudaMemcpyAsync(c->h_img.p, images_host, ib, cudaMemcpyHostToDevice, s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  rc = run_precompute(c, n_views, (const double*)c->h_P.p, (const float*)c->h_img.p, W, H, n_alpha, n_s, ECC_F32,
                      c->h_sino.p, nullptr, s, ready.ev.empty() ? nullptr : ready.ev.data());
  if (rc != ECC_OK) return rc;
  rc = run_evaluate(c, n_views, (const double*)c->h_P.p, nullptr, c->h_sino.p, nullptr, W, H, n_alpha, n_s, ECC_F32,
                    n_kappa, cauchy_c, nullptr, (int)np, (double*)c->h_total.p, nullptr, nullptr, nullptr, nullptr, false,
                    s);
  if (rc != ECC_OK) return rc;
  e = cudaMemcpyAsync(total_host, c->h_total.p, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  return ECC_OK;
}

int ecc_job_footprint(const ecc_job* job, size_t* bytes) {
  if (!bytes) return fail(nullptr, ECC_EINVAL, "bytes is NULL");
  std::string why;
  const int rc = ecc::serve_footprint(job, bytes, &why);
  if (rc != ECC_OK) return fail(nullptr, rc, "%s", why.c_str());
  return ECC_OK;
}

int ecc_submit(ecc_ctx* c, const ecc_job* job, uint64_t* ticket) {
  if (!c) return fail(nullptr, ECC_EINVAL, "ctx is NULL");
  std::string why;
  if (!c->serve) {
    DeviceGuard g(c->device);
    c->serve = ecc::serve_create(c->device, c->budget, &why);
    if (!c->serve) return fail(c, ECC_ECUDA, "%s", why.c_str());
  }
  const int rc = ecc::serve_submit(c->serve, job, ticket, &why);
  if (rc != ECC_OK) return fail(c, rc, "%s", why.c_str());
  return ECC_OK;
}

int ecc_poll(ecc_ctx* c, uint64_t ticket, ecc_result* out) {
  if (!c) return fail(nullptr, ECC_EINVAL, "ctx is NULL");
  if (!c->serve) return fail(c, ECC_EINVAL, "no job was submitted on this context");
  std::string why;
  const int rc = ecc::serve_poll(c->serve, ticket, out, &why);
  if (rc < 0) return fail(c, rc, "%s", why.c_str());
  return rc;
}

int ecc_serve_stats(ecc_ctx* c, long long* rounds, long long* job_rounds, int* max_batch, long long* line_pairs) {
  if (!c) return fail(nullptr, ECC_EINVAL, "ctx is NULL");
  if (!c->serve) {
    if (rounds) *rounds = 0;
    if (job_rounds) *job_rounds = 0;
    if (max_batch) *max_batch = 0;
    if (line_pairs) *line_pairs = 0;
    return ECC_OK;
  }
  ecc::serve_stats(c->serve, rounds, job_rounds, max_batch, line_pairs);
  return ECC_OK;
}

int ecc_serve_times(ecc_ctx* c, double* upload_ms, double* precompute_ms, double* round_ms) {
  if (!c) return fail(nullptr, ECC_EINVAL, "ctx is NULL");
  if (!c->serve) {
    if (upload_ms) *upload_ms = 0.0;
    if (precompute_ms) *precompute_ms = 0.0;
    if (round_ms) *round_ms = 0.0;
    return ECC_OK;
  }
  ecc::serve_times(c->serve, upload_ms, precompute_ms, round_ms);
  return ECC_OK;
}

}  // extern "C"

// Internal (tests and diagnostics only, not part of the public ABI): copies the
// first n view records and pair records of the last evaluation to host memory.
extern "C" int ecc_internal_dump(ecc_ctx* c, void* stream, int n_views, int n_pairs, void* views_out,
                                 void* pairs_out) {
  if (!c) return ECC_EINVAL;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && n_views > 0 && views_out && c->views.p)
    e = cudaMemcpy(views_out, c->views.p, sizeof(ecc::ViewRec) * (size_t)n_views, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && n_pairs > 0 && pairs_out && c->pairs.p)
    e = cudaMemcpy(pairs_out, c->pairs.p, sizeof(ecc::PairRec) * (size_t)n_pairs, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? ECC_OK : cuda_fail(c, e, "dump");
}

extern "C" int ecc_internal_record_sizes(int* view_bytes, int* pair_bytes) {
  *view_bytes = (int)sizeof(ecc::ViewRec);
  *pair_bytes = (int)sizeof(ecc::PairRec);
  return 0;
}
