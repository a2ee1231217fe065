// Internal device-side records and helpers of the ECC library (not part of the ABI).
//
// Data layout in device memory
//   P            [n_views][12]  FP64, row-major 3x4, world mm -> pixel homogeneous
//   sinogram     [n_views][n_alpha][n_s]  FP32 (alpha-major, rows contiguous in s)
//   ViewRec      [n_views]      FP64 per-view set-up (K0), with double-float copies
//   PairRec      [n_pairs]      double-float/int per-pair set-up (pair set-up kernel)
//   per-pair out {d, e} FP64 + N_kappa int32
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ecc {


// Per-view set-up (FP64).  P is scaled so that the third row of M has unit norm
// and det M > 0 (orientation-free: l = cof(M) n is invariant to P -> sP).
struct ViewRec {
  double P[12];    // normalised, after the view's rigid motion
  double C[3];     // source position (meet of the three rows of P)
  double up[3];    // unit detector up axis m3 x m1
  double cofc[9];  // cofactor matrix of M, rows; third row re-expressed for
                   // detector coordinates centred at ((W-1)/2, (H-1)/2)
  double u0, v0, D;  // principal point and source-detector distance [px]
  float qdf[30];     // C, up, cofc (15 values) as double-float (hi, lo) pairs, for the
                     // per-pair set-up on the FP32 pipes
  int status;        // 0 ok, 1 degenerate P
  int pad;
};

// Tangents of the per-view geometry with respect to the view's motion theta (6).
struct ViewTan {
  double dC[3][6];
  double dup[3][6];
  double dcofc[9][6];
};

// Tangents of the per-view quantities a pair reads, q = (C[3], up[3], cofc[9]), with
// respect to the 12 entries of the view's (unmoved) projection matrix P.
struct ViewTanP {
  double d[15][12];
};

// Per-pair set-up (double-float maps, integer sample ranges).
struct PairRec {
  float Af[2][12];  // per view (a, b): l_centred(kappa) = A (cos kappa, sin kappa), A 3x2 row-major,
                    // each entry a double-float pair (hi, lo)
  float dk_hi, dk_lo;  // Delta kappa as a double-float pair
  double c0[2];     // direction of the first sample, (k + 1/2) = 1/2, in the (w, v) frame
  double dk;        // Delta kappa
  int32_t a, b;     // view indices
  int32_t r0lo, r0hi, r1lo, r1hi;  // valid samples: [r0lo, r0hi) U [r1lo, r1hi)
  int32_t nk;       // N_kappa (number of valid samples)
  int32_t status;   // 0 ok, 1 degenerate pair (coincident sources / degenerate view)
};

// Device status bits (sticky per context until read).
enum : int {
  kStatusDegenerateView = 1,
  kStatusDegeneratePair = 2,
  kStatusNonfinitePair = 4,  // a pair's sum (or its gradient) was not finite: zeroed
};

// A unit direction (x, y) split into double-float pairs: (hi.x, hi.y, lo.x, lo.y).
// Layout of the tile-centre directions and of the alpha-row directions.
__host__ __device__ inline float4 split_dir(double x, double y) {
  const float hx = (float)x, hy = (float)y;
  return make_float4(hx, hy, (float)(x - (double)hx), (float)(y - (double)hy));
}

__host__ __device__ inline void pair_from_index(long long p, int n_views, int* a, int* b) {
  // row-major upper-triangular enumeration of a < b
  long long lo = 0;
  int aa = 0;
  // closed form: a = largest a with a*(2n-a-1)/2 <= p
  double n = (double)n_views;
  double disc = (2.0 * n - 1.0) * (2.0 * n - 1.0) - 8.0 * (double)p;
  aa = (int)floor(((2.0 * n - 1.0) - sqrt(disc > 0 ? disc : 0.0)) * 0.5);
  if (aa < 0) aa = 0;
  if (aa > n_views - 2) aa = n_views - 2;
  for (int it = 0; it < 3; ++it) {  // guard against rounding of the closed form
    lo = (long long)aa * (2LL * n_views - aa - 1) / 2;
    if (lo > p) { --aa; continue; }
    long long next = (long long)(aa + 1) * (2LL * n_views - aa - 2) / 2;
    if (next <= p) { ++aa; continue; }
    break;
  }
  lo = (long long)aa * (2LL * n_views - aa - 1) / 2;
  *a = aa;
  *b = (int)(aa + 1 + (p - lo));
}

}  // namespace ecc
