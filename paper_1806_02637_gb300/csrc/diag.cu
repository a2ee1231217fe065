// Internal diagnostic (not part of the public ABI): the L2 read rate that the
// gather kernels' L2 fractions are quoted against.  A grid of 8 blocks per SM
// reads a buffer small enough to stay resident in L2 with 16-byte loads that skip
// L1 (ld.global.cg), over and over (about 1 GB per launch, so that launch gaps do
// not count); the rate is bytes read over the CUDA-event time of `reps` back-to-back
// launches.  It allocates its buffer (a diagnostic, run once by the benchmark, not on
// the evaluation path).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ecc.h"

namespace {

__global__ void __launch_bounds__(256) l2_read_kernel(const float4* __restrict__ p, size_t n4, int passes,
                                                      float* __restrict__ sink) {
  float acc = 0.0f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < passes; ++r)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(p + i);
      acc += (v.x + v.y) + (v.z + v.w);
    }
  if (acc == 1.2345e-30f) sink[0] = acc;  // keeps the loads; never true for the zero buffer
}

}  // namespace

// *gbs = L2 read rate in GB/s over a resident buffer of `bytes` (multiple of 16),
// `reps` launches timed with CUDA events on the current device.
extern "C" int ecc_internal_l2_read_rate(size_t bytes, int reps, double* gbs) {
  if (!gbs || bytes < 16 || bytes % 16 != 0 || reps < 1) return ECC_EINVAL;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ECC_ECUDA;
  void* buf = nullptr;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = ECC_ECUDA;
  if (cudaMalloc(&buf, bytes) == cudaSuccess && cudaMalloc(&sink, sizeof(float)) == cudaSuccess &&
      cudaMemset(buf, 0, bytes) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess) {
    const size_t n4 = bytes / 16;
    const unsigned grid = 8u * (unsigned)n_sm;
    // each launch reads the buffer often enough (about 1 GB) that launch gaps do not count
    const int passes = (int)std::max<size_t>(1, ((size_t)1 << 30) / bytes);
    for (int i = 0; i < 3; ++i) l2_read_kernel<<<grid, 256>>>((const float4*)buf, n4, passes, sink);
    cudaEventRecord(e0);
    for (int i = 0; i < reps; ++i) l2_read_kernel<<<grid, 256>>>((const float4*)buf, n4, passes, sink);
    cudaEventRecord(e1);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f) {
      *gbs = (double)bytes * passes * reps / (ms * 1e-3) / 1e9;
      rc = ECC_OK;
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (buf) cudaFree(buf);
  return rc;
}
