// Per-view and per-pair FP64 set-up of the ECC path (no matrix inverse anywhere).
//
//  view_setup_kernel  one thread per view: rigid motion P' = P T(theta), scaling,
//                     source as the meet of the rows of P (Eq. 4/5), cofactor
//                     matrix, intrinsics.
//  pair_setup_kernel  one thread per pair: pencil frame around the baseline, the
//                     3x2 maps kappa -> epipolar line (the inverse-free form of
//                     Eq. 13/14), valid arcs from the detector corners, the sampled
//                     arc, the integer ranges of valid samples and the direction of
//                     each 32-sample tile centre.
#include "ecc_internal.cuh"
#include "kernels.cuh"

namespace ecc {

namespace {

__device__ inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// P T(theta), T = [R t; 0 1], R = Rz(rz) Ry(ry) Rx(rx).
__device__ void moved_projection(const double* P, const double* th, double* out) {
  double sx, cx, sy, cy, sz, cz;
  sincos(th[0], &sx, &cx);
  sincos(th[1], &sy, &cy);
  sincos(th[2], &sz, &cz);
  // R = Rz Ry Rx written out
  const double R[9] = {cz * cy, cz * sy * sx - sz * cx, cz * sy * cx + sz * sx,
                       sz * cy, sz * sy * sx + cz * cx, sz * sy * cx - cz * sx,
                       -sy,     cy * sx,                cy * cx};
  for (int i = 0; i < 3; ++i) {
    const double* p = P + 4 * i;
    for (int j = 0; j < 3; ++j) out[4 * i + j] = p[0] * R[j] + p[1] * R[3 + j] + p[2] * R[6 + j];
    out[4 * i + 3] = p[0] * th[3] + p[1] * th[4] + p[2] * th[5] + p[3];
  }
}

}  // namespace

__global__ void view_setup_kernel(int n_views, const double* __restrict__ P, const double* __restrict__ motion,
                                  int W, int H, ViewRec* __restrict__ out, int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_views) return;
  double Pm[12];
  if (motion) {
    moved_projection(P + 12 * i, motion + 6 * i, Pm);
  } else {
    for (int k = 0; k < 12; ++k) Pm[k] = P[12 * i + k];
  }
  ViewRec r;
  r.status = 0;
  r.pad = 0;
  double m1[3] = {Pm[0], Pm[1], Pm[2]}, m2[3] = {Pm[4], Pm[5], Pm[6]}, m3[3] = {Pm[8], Pm[9], Pm[10]};
  double c23[3];
  cross3(m2, m3, c23);
  const double det = dot3(m1, c23);
  const double n3 = sqrt(dot3(m3, m3));
  bool ok = isfinite(det) && isfinite(n3) && det != 0.0 && n3 > 0.0;
  const double sc = ok ? copysign(1.0, det) / n3 : 0.0;
  for (int k = 0; k < 12; ++k) r.P[k] = Pm[k] * sc;
  // source: meet of the first two rows (Pluecker, Eq. 4), then the point where that
  // line meets the third row, x = L_K P3 (Eq. 5 with p entering with opposite sign)
  const double* a = r.P;
  const double* b = r.P + 4;
  const double* c = r.P + 8;
  const double p_ = a[2] * b[3] - a[3] * b[2], q_ = a[1] * b[3] - a[3] * b[1], r_ = a[1] * b[2] - a[2] * b[1];
  const double s_ = a[0] * b[3] - a[3] * b[0], t_ = a[0] * b[2] - a[2] * b[0], u_ = a[0] * b[1] - a[1] * b[0];
  const double X0 = p_ * c[1] - q_ * c[2] + r_ * c[3];
  const double X1 = -p_ * c[0] + s_ * c[2] - t_ * c[3];
  const double X2 = q_ * c[0] - s_ * c[1] + u_ * c[3];
  const double X3 = -r_ * c[0] + t_ * c[1] - u_ * c[2];
  ok = ok && X3 != 0.0;
  const double iw = ok ? 1.0 / X3 : 0.0;
  r.C[0] = X0 * iw;
  r.C[1] = X1 * iw;
  r.C[2] = X2 * iw;
  double n1[3] = {r.P[0], r.P[1], r.P[2]}, n2[3] = {r.P[4], r.P[5], r.P[6]}, nn3[3] = {r.P[8], r.P[9], r.P[10]};
  double up[3];
  cross3(nn3, n1, up);
  const double nu = sqrt(dot3(up, up));
  ok = ok && nu > 0.0;
  for (int k = 0; k < 3; ++k) r.up[k] = ok ? up[k] / nu : 0.0;
  // cofactor rows: m2 x m3, m3 x m1, m1 x m2 (l = cof(M) n), third row moved to
  // detector coordinates centred at ((W-1)/2, (H-1)/2)
  double k0[3], k1[3], k2[3];
  cross3(n2, nn3, k0);
  cross3(nn3, n1, k1);
  cross3(n1, n2, k2);
  const double cx = 0.5 * (W - 1), cy = 0.5 * (H - 1);
  for (int k = 0; k < 3; ++k) {
    r.cofc[k] = k0[k];
    r.cofc[3 + k] = k1[k];
    r.cofc[6 + k] = cx * k0[k] + cy * k1[k] + k2[k];
  }
  r.u0 = dot3(n1, nn3);
  r.v0 = dot3(n2, nn3);
  const double dd = dot3(n1, n1) - r.u0 * r.u0;
  ok = ok && dd > 0.0;
  r.D = ok ? sqrt(dd) : 0.0;
  for (int k = 0; k < 3; ++k) ok = ok && isfinite(r.C[k]);
  if (!ok) {
    r.status = 1;
    atomicOr(status, kStatusDegenerateView);
  }
  out[i] = r;
}

namespace {

// Valid arc of the pencil for one view: the plane at kappa (c = (cos, sin)) meets
// the detector rectangle iff the values g_c . c at the four corners do not all have
// the same strict sign, g_c = A^T x_c.  If the g_c lie in a half plane (epipole
// outside), the valid directions (mod pi) run counter-clockwise from rot90(g_min)
// over the angle between the extreme g's; otherwise every plane is valid.
__device__ void view_arc(const double* A, int W, int H, double* clo, double* len) {
  const double xs[4] = {-0.5 * W, 0.5 * W, 0.5 * W, -0.5 * W};
  const double ys[4] = {-0.5 * H, -0.5 * H, 0.5 * H, 0.5 * H};
  double g[4][2];
  bool degenerate = false;
  for (int c = 0; c < 4; ++c) {
    g[c][0] = A[0] * xs[c] + A[2] * ys[c] + A[4];
    g[c][1] = A[1] * xs[c] + A[3] * ys[c] + A[5];
    const double n2 = g[c][0] * g[c][0] + g[c][1] * g[c][1];
    const double sc = A[0] * A[0] + A[1] * A[1] + A[2] * A[2] + A[3] * A[3] + A[4] * A[4] + A[5] * A[5];
    if (!(n2 > 1e-28 * sc)) degenerate = true;
  }
  int imin = -1, imax = -1;
  for (int i = 0; i < 4 && !degenerate; ++i) {
    bool is_min = true, is_max = true;
    for (int j = 0; j < 4; ++j) {
      if (g[i][0] * g[j][1] - g[i][1] * g[j][0] < 0.0) is_min = false;
      if (g[j][0] * g[i][1] - g[j][1] * g[i][0] < 0.0) is_max = false;
    }
    if (is_min && imin < 0) imin = i;
    if (is_max && imax < 0) imax = i;
  }
  if (degenerate || imin < 0 || imax < 0) {
    clo[0] = 0.0;
    clo[1] = -1.0;
    *len = kPi;
    return;
  }
  const double cr = g[imin][0] * g[imax][1] - g[imin][1] * g[imax][0];
  const double dt = g[imin][0] * g[imax][0] + g[imin][1] * g[imax][1];
  double phi = atan2(cr, dt);
  if (phi < 0.0) phi = 0.0;
  const double ng = sqrt(g[imin][0] * g[imin][0] + g[imin][1] * g[imin][1]);
  clo[0] = -g[imin][1] / ng;
  clo[1] = g[imin][0] / ng;
  *len = phi;
}

}  // namespace

__global__ void pair_setup_kernel(int n_views, long long n_pairs, const int32_t* __restrict__ pairs,
                                  const ViewRec* __restrict__ views, int W, int H, int K,
                                  PairRec* __restrict__ out, double2* __restrict__ ctile, int n_tiles,
                                  int* __restrict__ status) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  int a, b;
  if (pairs) {
    a = pairs[2 * p];
    b = pairs[2 * p + 1];
  } else {
    pair_from_index(p, n_views, &a, &b);
  }
  PairRec r;
  const bool in_range = a >= 0 && b >= 0 && a < n_views && b < n_views;
  if (!in_range) {  // caller's pair list names a view that does not exist
    a = 0;
    b = 0;
  }
  r.a = a;
  r.b = b;
  r.status = 0;
  r.r0lo = r.r0hi = r.r1lo = r.r1hi = 0;
  r.nk = 0;
  r.dk = 0.0;
  r.c0[0] = 1.0;
  r.c0[1] = 0.0;
  r.rot[0] = 1.0;
  r.rot[1] = 0.0;
  for (int i = 0; i < 12; ++i) (&r.A[0][0])[i] = 0.0;
  const ViewRec& va = views[a];
  const ViewRec& vb = views[b];
  double d[3] = {vb.C[0] - va.C[0], vb.C[1] - va.C[1], vb.C[2] - va.C[2]};
  const double nd = sqrt(dot3(d, d));
  bool ok = in_range && va.status == 0 && vb.status == 0 && nd > 0.0 && a != b;
  double u[3] = {0, 0, 0}, w[3] = {0, 0, 0}, v[3] = {0, 0, 0};
  if (ok) {
    for (int k = 0; k < 3; ++k) u[k] = d[k] / nd;
    double rr[3] = {va.up[0] + vb.up[0], va.up[1] + vb.up[1], va.up[2] + vb.up[2]};
    const double ru = dot3(rr, u);
    for (int k = 0; k < 3; ++k) w[k] = rr[k] - ru * u[k];
    double nw = sqrt(dot3(w, w));
    if (nw < 1e-6) {  // up_a + up_b along the baseline: world axis least aligned with u
      int ax = 0;
      double best = fabs(u[0]);
      for (int k = 1; k < 3; ++k)
        if (fabs(u[k]) < best) { best = fabs(u[k]); ax = k; }
      const double ui = u[ax];
      for (int k = 0; k < 3; ++k) w[k] = (k == ax ? 1.0 : 0.0) - ui * u[k];
      nw = sqrt(dot3(w, w));
    }
    for (int k = 0; k < 3; ++k) w[k] /= nw;
    cross3(w, u, v);
    const ViewRec* vv[2] = {&va, &vb};
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < 3; ++i) {
        r.A[s][2 * i + 0] = dot3(vv[s]->cofc + 3 * i, w);
        r.A[s][2 * i + 1] = dot3(vv[s]->cofc + 3 * i, v);
      }
    double clo[2][2], len[2];
    view_arc(r.A[0], W, H, clo[0], &len[0]);
    view_arc(r.A[1], W, H, clo[1], &len[1]);
    const int sv = len[0] <= len[1] ? 0 : 1;  // sample the shorter arc (ties: view a)
    const int ov = 1 - sv;
    const double dk = len[sv] / K;
    r.dk = dk;
    double sh, ch;
    sincos(0.5 * dk, &sh, &ch);
    r.c0[0] = ch * clo[sv][0] - sh * clo[sv][1];
    r.c0[1] = sh * clo[sv][0] + ch * clo[sv][1];
    sincos(dk, &r.rot[1], &r.rot[0]);
    // valid samples of the other view: y_k = delta0 + (k + 1/2) dk, valid iff
    // y_k <= len_o or pi <= y_k <= pi + len_o (angles mod pi from its arc start)
    if (len[ov] >= kPi) {
      r.r0lo = 0;
      r.r0hi = K;
      r.r1lo = r.r1hi = K;
    } else if (dk > 0.0) {
      double d0 = atan2(clo[ov][0] * clo[sv][1] - clo[ov][1] * clo[sv][0],
                        clo[ov][0] * clo[sv][0] + clo[ov][1] * clo[sv][1]);
      if (d0 < 0.0) d0 += kPi;
      if (d0 >= kPi) d0 -= kPi;
      const double e0 = floor((len[ov] - d0) / dk - 0.5);
      const double s1 = ceil((kPi - d0) / dk - 0.5);
      const double e1 = floor((kPi + len[ov] - d0) / dk - 0.5);
      int hi0 = (int)fmin(fmax(e0 + 1.0, 0.0), (double)K);
      int lo1 = (int)fmin(fmax(s1, (double)hi0), (double)K);
      int hi1 = (int)fmin(fmax(e1 + 1.0, (double)lo1), (double)K);
      r.r0lo = 0;
      r.r0hi = hi0;
      r.r1lo = lo1;
      r.r1hi = hi1;
    }
    r.nk = (r.r0hi - r.r0lo) + (r.r1hi - r.r1lo);
    // directions of the tile centres: (32 t + 16) dk from the arc start
    double s16, c16, s32, c32;
    sincos(16.0 * dk, &s16, &c16);
    sincos(32.0 * dk, &s32, &c32);
    double cx0 = c16 * clo[sv][0] - s16 * clo[sv][1];
    double cy0 = s16 * clo[sv][0] + c16 * clo[sv][1];
    double2* ct = ctile + p * n_tiles;
    for (int t = 0; t < n_tiles; ++t) {
      ct[t] = make_double2(cx0, cy0);
      const double nx = c32 * cx0 - s32 * cy0;
      const double ny = s32 * cx0 + c32 * cy0;
      cx0 = nx;
      cy0 = ny;
    }
  }
  if (!ok) {
    r.status = 1;
    atomicOr(status, kStatusDegeneratePair);
  }
  out[p] = r;
}

// Row directions (cos, sin)(m pi / n_alpha) in FP64 for the anchor look-ups.
__global__ void alpha_dir_kernel(int n_alpha, double2* __restrict__ dir) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_alpha) return;
  double s, c;
  sincospi((double)m / (double)n_alpha, &s, &c);
  dir[m] = make_double2(c, s);
}

}  // namespace ecc
