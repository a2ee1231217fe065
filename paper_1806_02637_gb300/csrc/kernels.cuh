// Kernel declarations shared by the translation units of the library.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>
#include "ecc_internal.cuh"

namespace ecc {

__global__ void view_setup_kernel(int n_views, const double* P, const double* motion, int W, int H, ViewRec* out,
                                  int* status);
// pairs [p_begin, p_end) of the row-major a < b enumeration (pairs == NULL) or of the list
__global__ void pair_setup_kernel(int n_views, long long p_begin, long long p_end, const int32_t* pairs,
                                  const ViewRec* views, int W, int H, int K, PairRec* out, float4* ctile, int n_tiles,
                                  int reuse_sampling, int* status);
__global__ void view_tangent_kernel(int n_views, const double* P, const double* motion, int W, int H, ViewTan* out);
__global__ void view_grad_theta_kernel(int n_views, long long n_pairs, const int32_t* pairs, const float2* gq,
                                       const ViewTan* vtan, double* grad);
__global__ void view_tangent_P_kernel(int n_views, const double* P, const double* motion, int W, int H,
                                      ViewTanP* out);
__global__ void pair_grad_q_kernel(long long n_pairs, const PairRec* prs, const ViewRec* views, const double* Gpp,
                                   float2* gq);
__global__ void view_grad_P_kernel(int n_views, long long n_pairs, const int32_t* pairs, const float2* gq,
                                   const ViewTanP* vtan, double* grad_P);
__global__ void alpha_dir_kernel(int n_alpha, float4* dir);

// Per (view, alpha-row) line parameters of the Joseph line sums (32.32 fixed point).
struct RadonRow {
  long long B0;    // coordinate along the interpolation axis at rho index 0, step 0
  long long STEP;  // per rho index
  long long DY;    // per step along the integration axis
  float inv_len;   // path length per step: 1/|cos a| (rows) or 1/|sin a| (columns)
  float ca, sa;    // cos, sin of alpha
  int rows_mode;   // 1: step over image rows, interpolate in x; 0: columns
};

struct RadonView {  // per-view weights (FP32 copies of the FP64 set-up)
  float u0, v0, D;
  int pad;
};

// Callbacks around every kernel launch (launch counting and optional CUDA-event
// timing by the context).
struct LaunchHooks {
  void (*begin)(void* ctx, const char* name, cudaStream_t s) = nullptr;
  void (*end)(void* ctx, const char* name, cudaStream_t s) = nullptr;
  void* ctx = nullptr;
  void on_begin(const char* n, cudaStream_t s) const {
    if (begin) begin(ctx, n, s);
  }
  void on_end(const char* n, cudaStream_t s) const {
    if (end) end(ctx, n, s);
  }
};

// Parameters of the pair kernel for one scan (device pointers).
struct PairArgs {
  long long n_pairs;
  const PairRec* prs;
  const float4* ctile;      // tile-centre directions (hi.x, hi.y, lo.x, lo.y)
  int n_tiles;
  const float4* alpha_dir;  // alpha-row directions (cos, sin as double-float pairs)
  const void* sino;
  const float* scales;  // FP16 storage only, else NULL
  int n_alpha, n_s, K;
  // grid constants (set by pair_args_grid): alpha rows per radian, s bins per pixel
  // (FP32 and as a double-float pair), and (n_s - 1) / 2 as a double-float pair
  float inv_dalpha, inv_ds_f, inv_ds_hi, inv_ds_lo, half_hi, half_lo;
  float cauchy_c;
  double* per_pair;
  int32_t* nk_out;
  double* block_partial;
  double* Gpp;  // adjoint output, NULL for the plain evaluation
  int* status;  // device status word (kStatus* bits OR-ed in), or NULL
};

inline void pair_args_grid(PairArgs& g, int n_alpha, int n_s, int W, int H) {
  const double inv_ds = (double)(n_s - 1) / std::sqrt((double)W * W + (double)H * H);
  const double inv_dalpha = (double)n_alpha / 3.14159265358979323846;
  const double half = 0.5 * (n_s - 1);
  g.n_alpha = n_alpha;
  g.n_s = n_s;
  g.inv_dalpha = (float)inv_dalpha;
  g.inv_ds_f = (float)inv_ds;
  g.inv_ds_hi = (float)inv_ds;
  g.inv_ds_lo = (float)(inv_ds - (double)g.inv_ds_hi);
  g.half_hi = (float)half;
  g.half_lo = (float)(half - (double)g.half_hi);
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_radon(const ViewRec* views, int n_views, const float* images, int W, int H, int n_alpha, int n_s,
                         int dtype, void* sino_out, float* scales_out, RadonRow* table, void* wimg, float* stage,
                         int batch_views, const LaunchHooks& hooks, cudaStream_t stream,
                         const cudaEvent_t* batch_ready = nullptr);  // per batch: wait before reading its images
size_t radon_f16_stage_bytes(int n_alpha, int n_s, int batch_views);
int radon_pad(int W, int H, int n_s);
// Bytes of one view's weighted-image planes (interpolation pairs, both orientations).
size_t radon_plane_bytes(int W, int H, int n_s);

cudaError_t launch_ecc_pairs(long long n_pairs, const PairRec* prs, const float4* ctile, int n_tiles,
                             const float4* alpha_dir, const void* sino, const float* scales, int dtype,
                             int n_alpha, int n_s, int K, int W, int H, double cauchy_c, double* per_pair, int32_t* nk_out,
                             double* block_partial, double* Gpp, int* status, int* n_blocks_out,
                             const LaunchHooks& hooks, cudaStream_t stream);

cudaError_t launch_reduce(const double* partial, int n, double* total, const LaunchHooks& hooks,
                          cudaStream_t stream);

// ---------------------------------------------------------------- serving rounds
// One active job of a serving round (device copy of the scheduler's table).  Every
// round evaluates each job's total and, with do_grad, its gradient and one step
// theta <- theta - step * grad.  The kernels below cover all jobs of a round; a
// flattened index (view, pair or pair block) is mapped to its job by binary search
// over the per-job prefix offsets (n_jobs + 1 entries each).
struct ServeJob {
  PairArgs pair;  // pair kernel parameters (block_partial and Gpp set, per_pair/nk_out NULL)
  int dtype;
  int n_views, W, H, n_tiles;
  int do_grad;
  double step;
  const double* P;   // [n_views][12]
  double* theta;     // [n_views][6]
  double* grad;      // [n_views][6]
  ViewRec* views;
  ViewTan* vtan;
  float2* gpp;        // [n_pairs][30] d e / d (C, up, cofc) of views a and b, double-float pairs
  double* total_out;  // this round's total
  int* status;
  // motion model: per-view (theta stepped directly) or Akima spline of node values
  int model, n_nodes, mask;  // mask: estimated parameters (bits 0..5)
  double h;                  // node spacing in views
  const double* theta0;      // [n_views][6] fixed part (motion0)
  double* nodes;             // [n_nodes][6]
  double* jac;               // [n_views][6][6] d theta / d nodes (local window)
  int* jbase;                // [n_views][6] first node of the window
};

__host__ __device__ inline int serve_job_of(const long long* off, int n_jobs, long long i) {
  int lo = 0, hi = n_jobs - 1;  // last job with off[j] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Per-view set-up and tangents; per-pair set-up.
cudaError_t launch_serve_setup(const ServeJob* jobs, const long long* voff, const long long* poff, int n_jobs,
                               long long n_views, long long n_pairs, cudaStream_t stream);
// Pair kernel over all jobs' pair blocks: a persistent grid that takes blocks from a
// counter (reset here), then each job's fixed-order total.
cudaError_t launch_serve_pairs(const ServeJob* jobs, const long long* boff, int n_jobs,
                               unsigned long long* counter, int grid, cudaStream_t stream);
int serve_pairs_blocks_per_sm();
// Motion of the round: theta = theta0 + spline(nodes) for spline jobs (and the
// window Jacobians); per-view jobs keep their theta.
cudaError_t launch_serve_motion(const ServeJob* jobs, const long long* voff, int n_jobs, long long n_views,
                                cudaStream_t stream);
// Pair gradients, per-view gradient sums and the gradient steps.
cudaError_t launch_serve_grad(const ServeJob* jobs, const long long* voff, const long long* poff, int n_jobs,
                              long long n_views, long long n_pairs, cudaStream_t stream);

}  // namespace ecc
