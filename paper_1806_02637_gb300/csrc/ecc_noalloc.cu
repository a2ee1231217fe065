// ecc_evaluate_noalloc: ecc_evaluate without a context and without any device
// allocation (declared in include/ecc.h).
//
// Some callers cannot allocate device memory once they are running: an application
// that hands all free device memory to its own pool at start-up (any later
// cudaMalloc fails), or a pipeline with a fixed memory budget where an allocation's
// implicit device synchronisation would stall other work.  This variant keeps its
// scratch (view and pair records, tile directions, alpha directions, per-block
// partial sums, status word) in one statically sized device array of this file,
// which the CUDA runtime places when the library's module is loaded, and it calls
// no allocator.  The price is fixed limits (below) and one scratch area shared by
// every call on a device: calls that overlap on the GPU (two streams, two host
// threads) race on it, so the caller serialises them, e.g. by using one stream.
//
// Set-up: every call looks up the array's device address with cudaGetSymbolAddress,
// with the caller's device current (a host-side lookup that allocates nothing).  The
// address is not cached: after cudaDeviceReset, or after another library in the
// process resets the primary context, the module is loaded again and the array may
// sit at a new address, and a cached one would then send the kernels to stale
// memory.  The first call on a device may load the library's module (lazy module
// loading), so make it outside any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "../../include/ecc.h"
#include "ecc_internal.cuh"
#include "kernels.cuh"

// The scratch array itself.  Its device address is only ever obtained through
// cudaGetSymbolAddress below; host code never uses the symbol as a pointer.
static __device__ __align__(256) unsigned char g_noalloc_scratch[size_t(5) << 20];

namespace {

// Limits of the static scratch (5 MiB).
constexpr int kMaxViews = 512;
constexpr int kMaxAlpha = 4096;
constexpr int kMaxPairs = 8192;
constexpr long long kMaxPairTiles = 131072;  // n_pairs * ceil(n_kappa / 32)
constexpr size_t kScratchBytes = sizeof(g_noalloc_scratch);

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Section offsets inside the array (each 256-byte aligned).
constexpr size_t kOffStatus = 0;
constexpr size_t kOffViews = align256(kOffStatus + sizeof(int));
constexpr size_t kOffAlpha = align256(kOffViews + sizeof(ecc::ViewRec) * kMaxViews);
constexpr size_t kOffPairs = align256(kOffAlpha + sizeof(float4) * kMaxAlpha);
constexpr size_t kOffPartial = align256(kOffPairs + sizeof(ecc::PairRec) * kMaxPairs);
constexpr size_t kOffPerPair = align256(kOffPartial + sizeof(double) * ((kMaxPairs + 7) / 8));
constexpr size_t kOffTiles = align256(kOffPerPair + sizeof(double) * 2 * kMaxPairs);
constexpr size_t kEnd = kOffTiles + sizeof(float4) * kMaxPairTiles;
static_assert(kEnd <= kScratchBytes, "no-alloc scratch layout exceeds the static array");

}  // namespace

extern "C" int ecc_evaluate_noalloc(int n_views, const double* P, const double* motion, const void* sino,
                                    const float* scales, int W, int H, int n_alpha, int n_s, int dtype, int n_kappa,
                                    double cauchy_c, const int32_t* pairs, int n_pairs, double* total,
                                    double* per_pair, int32_t* nkappa, void* stream, char* err, size_t err_len) {
  auto fail = [err, err_len](int code, const char* text) {
    if (err && err_len > 0) std::snprintf(err, err_len, "%s", text);
    return code;
  };
  if (err && err_len > 0) err[0] = '\0';
  char msg[256];
  if (!P || !sino || !total) return fail(ECC_EINVAL, "P, sino or total is NULL");
  if (n_views < 1 || n_views > kMaxViews) {
    std::snprintf(msg, sizeof msg, "n_views %d outside [1, %d] of the no-alloc scratch", n_views, kMaxViews);
    return fail(ECC_EINVAL, msg);
  }
  if (W < 2 || H < 2 || W > 16384 || H > 16384) return fail(ECC_EINVAL, "detector size out of range");
  if (n_alpha < 4 || n_alpha > kMaxAlpha) {
    std::snprintf(msg, sizeof msg, "n_alpha %d outside [4, %d] of the no-alloc scratch", n_alpha, kMaxAlpha);
    return fail(ECC_EINVAL, msg);
  }
  if (n_s < 2 || n_s > 65535) return fail(ECC_EINVAL, "n_s out of range [2, 65535]");
  if (dtype != ECC_F32 && dtype != ECC_F16 && dtype != ECC_BF16) return fail(ECC_EINVAL, "unknown dtype");
  if (dtype == ECC_F16 && !scales) return fail(ECC_EINVAL, "ECC_F16 needs scales");
  if (n_kappa < 1 || n_kappa > 65536) return fail(ECC_EINVAL, "n_kappa out of range [1, 65536]");
  if (n_pairs < 0 || n_pairs > kMaxPairs) {
    std::snprintf(msg, sizeof msg, "n_pairs %d outside [0, %d] of the no-alloc scratch", n_pairs, kMaxPairs);
    return fail(ECC_EINVAL, msg);
  }
  const int n_tiles = (n_kappa + 31) / 32;
  if ((long long)n_pairs * n_tiles > kMaxPairTiles) {
    std::snprintf(msg, sizeof msg, "n_pairs * ceil(n_kappa / 32) = %lld exceeds %lld of the no-alloc scratch",
                  (long long)n_pairs * n_tiles, kMaxPairTiles);
    return fail(ECC_EINVAL, msg);
  }
  if (!pairs && n_pairs > 0 && (long long)n_views * (n_views - 1) / 2 != n_pairs)
    return fail(ECC_EINVAL, "pairs is NULL but n_pairs != n_views (n_views - 1) / 2");
  if (!std::isfinite(cauchy_c)) return fail(ECC_EINVAL, "cauchy_c is not finite");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ECC_ECUDA, "no usable current CUDA device");
  // the array's address in the current device's context, looked up on every call
  unsigned char* base = nullptr;
  {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the no-alloc scratch: %s", cudaGetErrorString(e));
      return fail(ECC_ECUDA, msg);
    }
    base = static_cast<unsigned char*>(p);
  }
  cudaStream_t s = (cudaStream_t)stream;
  int* status = reinterpret_cast<int*>(base + kOffStatus);
  ecc::ViewRec* views = reinterpret_cast<ecc::ViewRec*>(base + kOffViews);
  float4* adir = reinterpret_cast<float4*>(base + kOffAlpha);
  ecc::PairRec* prs = reinterpret_cast<ecc::PairRec*>(base + kOffPairs);
  double* partial = reinterpret_cast<double*>(base + kOffPartial);
  float4* ctile = reinterpret_cast<float4*>(base + kOffTiles);
  if (!per_pair) per_pair = reinterpret_cast<double*>(base + kOffPerPair);

  if (n_pairs == 0) {
    e = cudaMemsetAsync(total, 0, sizeof(double), s);
    return e == cudaSuccess ? ECC_OK : fail(ECC_ECUDA, cudaGetErrorString(e));
  }
  // the status word is OR-accumulated by the kernels: start it at zero
  e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e != cudaSuccess) return fail(ECC_ECUDA, cudaGetErrorString(e));
  const ecc::LaunchHooks hk;  // no context: nothing to count or time
  ecc::view_setup_kernel<<<(n_views + 127) / 128, 128, 0, s>>>(n_views, P, motion, W, H, views, status);
  ecc::alpha_dir_kernel<<<(n_alpha + 255) / 256, 256, 0, s>>>(n_alpha, adir);
  ecc::pair_setup_kernel<<<(n_pairs + 127) / 128, 128, 0, s>>>(n_views, 0, n_pairs, pairs, views, W, H, n_kappa, prs,
                                                               ctile, n_tiles, 0, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(ECC_ECUDA, cudaGetErrorString(e));
  int nb = 0;
  e = ecc::launch_ecc_pairs(n_pairs, prs, ctile, n_tiles, adir, sino, scales, dtype, n_alpha, n_s, n_kappa, W, H,
                            cauchy_c, per_pair, nkappa, partial, nullptr, status, &nb, hk, s);
  if (e != cudaSuccess) return fail(ECC_ECUDA, cudaGetErrorString(e));
  e = ecc::launch_reduce(partial, nb, total, hk, s);
  if (e != cudaSuccess) return fail(ECC_ECUDA, cudaGetErrorString(e));
  return ECC_OK;
}
