// Per-view and per-pair set-up of the ECC path (no matrix inverse anywhere): FP64 per
// view, double-float (about 48 bits, on the FP32 pipes) per pair.
//
//  view_setup_kernel  one thread per view: rigid motion P' = P T(theta), scaling,
//                     source as the meet of the rows of P (Eq. 4/5), cofactor
//                     matrix, intrinsics.
//  pair_setup_kernel  one thread per pair: pencil frame around the baseline, the
//                     3x2 maps kappa -> epipolar line (the inverse-free form of
//                     Eq. 13/14), valid arcs from the detector corners, the sampled
//                     arc, the integer ranges of valid samples and the direction of
//                     each 32-sample tile centre.
#include "df.cuh"
#include "dual.cuh"
#include "motion.cuh"
#include "ecc_internal.cuh"
#include "kernels.cuh"

namespace ecc {

namespace {

template <class T>
__host__ __device__ inline void cross3(const T* a, const T* b, T* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
template <class T>
__host__ __device__ inline T dot3(const T* a, const T* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__host__ __device__ inline void sc_pair(double x, double* s, double* c) { sincos(x, s, c); }
template <int N>
__device__ inline void sc_pair(const Dual<N>& x, Dual<N>* s, Dual<N>* c) { sincos(x, s, c); }

// P T(theta), T = [R t; 0 1], R = Rz(rz) Ry(ry) Rx(rx).
template <class TP, class T>
__host__ __device__ void moved_projection(const TP* P, const T* th, T* out) {
  T sx, cx, sy, cy, sz, cz;
  sc_pair(th[0], &sx, &cx);
  sc_pair(th[1], &sy, &cy);
  sc_pair(th[2], &sz, &cz);
  const T R[9] = {cz * cy, cz * sy * sx - sz * cx, cz * sy * cx + sz * sx,
                  sz * cy, sz * sy * sx + cz * cx, sz * sy * cx - cz * sx,
                  -sy,     cy * sx,                cy * cx};
  for (int i = 0; i < 3; ++i) {
    const TP* p = P + 4 * i;
    for (int j = 0; j < 3; ++j) out[4 * i + j] = p[0] * R[j] + p[1] * R[3 + j] + p[2] * R[6 + j];
    out[4 * i + 3] = p[0] * th[3] + p[1] * th[4] + p[2] * th[5] + T(p[3]);
  }
}

// Per-view geometry from a (moved) projection matrix: scaled P (third row of M
// unit, det M > 0), source as the meet of the rows (Eq. 4, then Eq. 5 with p
// entering with the opposite sign), up axis m3 x m1, cofactor rows (m2 x m3,
// m3 x m1, m1 x m2; l = cof(M) n) with the third row for centred detector
// coordinates, principal point and source-detector distance.  Returns false for
// a degenerate P.
template <class T>
__host__ __device__ bool view_geometry(const T* Pm, int W, int H, T* Pn, T* C, T* up, T* cofc, T* u0, T* v0, T* D) {
  T m1[3] = {Pm[0], Pm[1], Pm[2]}, m2[3] = {Pm[4], Pm[5], Pm[6]}, m3[3] = {Pm[8], Pm[9], Pm[10]};
  T c23[3];
  cross3(m2, m3, c23);
  const T det = dot3(m1, c23);
  const T n3 = sqrt(dot3(m3, m3));
  bool ok = isfinite(value(det)) && isfinite(value(n3)) && value(det) != 0.0 && value(n3) > 0.0;
  for (int k = 0; k < 12; ++k) ok = ok && isfinite(value(Pm[k]));  // NaN / Inf anywhere, the motion's included
  const T sc = ok ? T(copysign(1.0, value(det))) / n3 : T(0.0);
  for (int k = 0; k < 12; ++k) Pn[k] = Pm[k] * sc;
  const T* a = Pn;
  const T* b = Pn + 4;
  const T* c = Pn + 8;
  const T p_ = a[2] * b[3] - a[3] * b[2], q_ = a[1] * b[3] - a[3] * b[1], r_ = a[1] * b[2] - a[2] * b[1];
  const T s_ = a[0] * b[3] - a[3] * b[0], t_ = a[0] * b[2] - a[2] * b[0], u_ = a[0] * b[1] - a[1] * b[0];
  const T X0 = p_ * c[1] - q_ * c[2] + r_ * c[3];
  const T X1 = -p_ * c[0] + s_ * c[2] - t_ * c[3];
  const T X2 = q_ * c[0] - s_ * c[1] + u_ * c[3];
  const T X3 = -r_ * c[0] + t_ * c[1] - u_ * c[2];
  ok = ok && value(X3) != 0.0;
  const T iw = ok ? T(1.0) / X3 : T(0.0);
  C[0] = X0 * iw;
  C[1] = X1 * iw;
  C[2] = X2 * iw;
  T n1[3] = {Pn[0], Pn[1], Pn[2]}, n2[3] = {Pn[4], Pn[5], Pn[6]}, nn3[3] = {Pn[8], Pn[9], Pn[10]};
  T upr[3];
  cross3(nn3, n1, upr);
  const T nu = sqrt(dot3(upr, upr));
  ok = ok && value(nu) > 0.0;
  for (int k = 0; k < 3; ++k) up[k] = ok ? upr[k] / nu : T(0.0);
  T k0[3], k1[3], k2[3];
  cross3(n2, nn3, k0);
  cross3(nn3, n1, k1);
  cross3(n1, n2, k2);
  const double cxd = 0.5 * (W - 1), cyd = 0.5 * (H - 1);
  for (int k = 0; k < 3; ++k) {
    cofc[k] = k0[k];
    cofc[3 + k] = k1[k];
    cofc[6 + k] = cxd * k0[k] + cyd * k1[k] + k2[k];
  }
  *u0 = dot3(n1, nn3);
  *v0 = dot3(n2, nn3);
  const T dd = dot3(n1, n1) - *u0 * *u0;
  ok = ok && value(dd) > 0.0;
  *D = ok ? sqrt(dd) : T(0.0);
  for (int k = 0; k < 3; ++k) ok = ok && isfinite(value(C[k]));
  return ok;
}

}  // namespace

__host__ __device__ ViewRec setup_view(const double* P, const double* motion, int W, int H) {
  double Pm[12];
  if (motion) {
    moved_projection(P, motion, Pm);
  } else {
    for (int k = 0; k < 12; ++k) Pm[k] = P[k];
  }
  ViewRec r;
  r.pad = 0;
  const bool ok = view_geometry(Pm, W, H, r.P, r.C, r.up, r.cofc, &r.u0, &r.v0, &r.D);
  r.status = ok ? 0 : 1;
  for (int k = 0; k < 15; ++k) {
    const df q = df_from_double(k < 3 ? r.C[k] : (k < 6 ? r.up[k - 3] : r.cofc[k - 6]));
    r.qdf[2 * k] = q.hi;
    r.qdf[2 * k + 1] = q.lo;
  }
  return r;
}

__global__ void view_setup_kernel(int n_views, const double* __restrict__ P, const double* __restrict__ motion,
                                  int W, int H, ViewRec* __restrict__ out, int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_views) return;
  const ViewRec r = setup_view(P + 12 * i, motion ? motion + 6 * i : nullptr, W, H);
  if (r.status) atomicOr(status, kStatusDegenerateView);
  out[i] = r;
}

// Tangents of the per-view geometry with respect to the view's own motion
// parameters (forward mode, FP64): d C / d theta, d up / d theta, d cofc / d theta.
__device__ ViewTan view_tangent(const double* P, const double* motion, int W, int H) {
  using D6 = Dual<6>;
  D6 th[6];
  for (int j = 0; j < 6; ++j) {
    th[j] = D6(motion ? motion[j] : 0.0);
    th[j].d[j] = 1.0;
  }
  D6 Pm[12], Pn[12], C[3], up[3], cofc[9], u0, v0, D;
  moved_projection(P, th, Pm);
  // a degenerate view's pairs carry no gradient; zero tangents keep its row at 0
  // (its NaN / Inf geometry would otherwise turn 0 x tangent into NaN)
  const double ok = view_geometry(Pm, W, H, Pn, C, up, cofc, &u0, &v0, &D) ? 1.0 : 0.0;
  ViewTan t;
  for (int j = 0; j < 6; ++j) {
    for (int k = 0; k < 3; ++k) {
      t.dC[k][j] = ok ? C[k].d[j] : 0.0;
      t.dup[k][j] = ok ? up[k].d[j] : 0.0;
    }
    for (int k = 0; k < 9; ++k) t.dcofc[k][j] = ok ? cofc[k].d[j] : 0.0;
  }
  return t;
}

// The same tangents, one thread per (view, motion parameter j): column j of the
// view's ViewTan (a single tangent direction, six times the threads of one Dual<6>
// per view).
__global__ void view_tangent_kernel(int n_views, const double* __restrict__ P, const double* __restrict__ motion,
                                    int W, int H, ViewTan* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6LL * n_views) return;
  const int lam = (int)(i / 6), j = (int)(i % 6);
  using D1 = Dual<1>;
  D1 th[6];
  for (int k = 0; k < 6; ++k) th[k] = D1(motion ? motion[6 * lam + k] : 0.0);
  th[j].d[0] = 1.0;
  D1 Pm[12], Pn[12], C[3], up[3], cofc[9], u0, v0, D;
  moved_projection(P + 12 * lam, th, Pm);
  // a degenerate view's pairs carry no gradient; zero tangents keep its row at 0
  const bool ok = view_geometry(Pm, W, H, Pn, C, up, cofc, &u0, &v0, &D);
  ViewTan& t = out[lam];
  for (int k = 0; k < 3; ++k) {
    t.dC[k][j] = ok ? C[k].d[0] : 0.0;
    t.dup[k][j] = ok ? up[k].d[0] : 0.0;
  }
  for (int k = 0; k < 9; ++k) t.dcofc[k][j] = ok ? cofc[k].d[0] : 0.0;
}

// Tangents of q = (C, up, cofc) with respect to the 12 entries of the unmoved P
// (forward mode, FP64; the view uses P T(theta)): one thread per (view, entry j),
// one tangent direction each.
__global__ void view_tangent_P_kernel(int n_views, const double* __restrict__ P, const double* __restrict__ motion,
                                      int W, int H, ViewTanP* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 12LL * n_views) return;
  const int lam = (int)(i / 12), j = (int)(i % 12);
  using D1 = Dual<1>;
  D1 Pd[12], Pm[12], Pn[12], C[3], up[3], cofc[9], u0, v0, D;
  for (int k = 0; k < 12; ++k) Pd[k] = D1(P[12 * lam + k]);
  Pd[j].d[0] = 1.0;
  if (motion) {
    D1 th[6];
    for (int k = 0; k < 6; ++k) th[k] = D1(motion[6 * lam + k]);
    moved_projection(Pd, th, Pm);
  } else {
    for (int k = 0; k < 12; ++k) Pm[k] = Pd[k];
  }
  const bool ok = view_geometry(Pm, W, H, Pn, C, up, cofc, &u0, &v0, &D);  // degenerate: zero tangents
  ViewTanP& t = out[lam];
  for (int k = 0; k < 3; ++k) {
    t.d[k][j] = ok ? C[k].d[0] : 0.0;
    t.d[3 + k][j] = ok ? up[k].d[0] : 0.0;
  }
  for (int k = 0; k < 9; ++k) t.d[6 + k][j] = ok ? cofc[k].d[0] : 0.0;
}

namespace {

// Double-float vector helpers of the per-pair set-up.
__host__ __device__ inline df qget(const ViewRec& v, int k) { return df{v.qdf[2 * k], v.qdf[2 * k + 1]}; }
__host__ __device__ inline df df_dot3(const df* a, const df* b) {
  return df_add(df_add(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
}
__host__ __device__ inline df df_cross2(df ax, df ay, df bx, df by) { return df_sub(df_mul(ax, by), df_mul(ay, bx)); }
__host__ __device__ inline df df_sel(bool c, df a, df b) { return c ? a : b; }

// Frame of the pencil of epipolar planes around the baseline C_a -> C_b, in
// double-float: u = baseline direction, w = (up_a + up_b) made orthogonal to u (below
// |w| = 1e-6 the world axis least aligned with u, the first within 1e-9 of the
// smallest |u_k| so that ties are not left to rounding), v = w x u; the plane at kappa
// has normal cos(kappa) w + sin(kappa) v.  Normalisations are products by reciprocal
// square roots.  Returns false for coincident sources.
__host__ __device__ bool pencil_frame_df(const ViewRec& va, const ViewRec& vb, df* w, df* v) {
  df d[3], rr[3], u[3];
  for (int k = 0; k < 3; ++k) {
    d[k] = df_sub(qget(vb, k), qget(va, k));
    rr[k] = df_add(qget(va, 3 + k), qget(vb, 3 + k));
  }
  const df nd2 = df_dot3(d, d);
  if (!(nd2.hi > 0.0f)) return false;
  const df ind = df_rsqrt(nd2);
  for (int k = 0; k < 3; ++k) u[k] = df_mul(d[k], ind);
  const df ru = df_dot3(rr, u);
  for (int k = 0; k < 3; ++k) w[k] = df_sub(rr[k], df_mul(ru, u[k]));
  df nw2 = df_dot3(w, w);
  if (nw2.hi < 1e-12f) {
    // the first axis within 1e-9 of the smallest |u_k|: ties are not left to rounding
    const double ua[3] = {fabs(df_to_double(u[0])), fabs(df_to_double(u[1])), fabs(df_to_double(u[2]))};
    const double best = fmin(ua[0], fmin(ua[1], ua[2]));
    const int ax = ua[0] <= best + 1e-9 ? 0 : (ua[1] <= best + 1e-9 ? 1 : 2);
    const df ui = ax == 0 ? u[0] : (ax == 1 ? u[1] : u[2]);
    for (int k = 0; k < 3; ++k) w[k] = df_sub(df{k == ax ? 1.0f : 0.0f, 0.0f}, df_mul(ui, u[k]));
    nw2 = df_dot3(w, w);
  }
  const df inw = df_rsqrt(nw2);
  for (int k = 0; k < 3; ++k) w[k] = df_mul(w[k], inw);
  v[0] = df_cross2(w[1], w[2], u[1], u[2]);
  v[1] = df_cross2(w[2], w[0], u[2], u[0]);
  v[2] = df_cross2(w[0], w[1], u[0], u[1]);
  return true;
}

// Reverse mode of pencil_frame_df (the same steps in double-float): given gw = d e / d w
// and gv = d e / d v, returns d e / d (Ca, Cb, up) in gCa, gCb and gup (the same for both
// up axes, which enter as their sum).  Each step's adjoint follows from its forward
// rule: v = w x u gives w' += u x v', u' += v' x w; y = x / |x| gives
// x' = (y' - (y'.y) y) / |x|; w_t = r - (r.u) u gives r' = w_t' - (w_t'.u) u and
// u' -= (w_t'.u) r + (r.u) w_t' (for the fallback axis e: u' -= (w_t'.u) e_ax + u_ax w_t').
__host__ __device__ bool pencil_frame_adjoint_df(const ViewRec& va, const ViewRec& vb, const df* gw, const df* gv,
                                                 df* w, df* v, df* gCa, df* gCb, df* gup) {
  df d[3], rr[3], u[3], wt[3];
  for (int k = 0; k < 3; ++k) {
    d[k] = df_sub(qget(vb, k), qget(va, k));
    rr[k] = df_add(qget(va, 3 + k), qget(vb, 3 + k));
  }
  const df nd2 = df_dot3(d, d);
  if (!(nd2.hi > 0.0f)) return false;
  const df ind = df_rsqrt(nd2);
  for (int k = 0; k < 3; ++k) u[k] = df_mul(d[k], ind);
  const df ru = df_dot3(rr, u);
  for (int k = 0; k < 3; ++k) wt[k] = df_sub(rr[k], df_mul(ru, u[k]));
  df nw2 = df_dot3(wt, wt);
  int ax = -1;
  if (nw2.hi < 1e-12f) {
    const double ua[3] = {fabs(df_to_double(u[0])), fabs(df_to_double(u[1])), fabs(df_to_double(u[2]))};
    const double best = fmin(ua[0], fmin(ua[1], ua[2]));
    ax = ua[0] <= best + 1e-9 ? 0 : (ua[1] <= best + 1e-9 ? 1 : 2);
    const df ui = ax == 0 ? u[0] : (ax == 1 ? u[1] : u[2]);
    for (int k = 0; k < 3; ++k) wt[k] = df_sub(df{k == ax ? 1.0f : 0.0f, 0.0f}, df_mul(ui, u[k]));
    nw2 = df_dot3(wt, wt);
  }
  const df inw = df_rsqrt(nw2);
  for (int k = 0; k < 3; ++k) w[k] = df_mul(wt[k], inw);
  v[0] = df_cross2(w[1], w[2], u[1], u[2]);
  v[1] = df_cross2(w[2], w[0], u[2], u[0]);
  v[2] = df_cross2(w[0], w[1], u[0], u[1]);
  // reverse
  df gwt_in[3], gu[3], gwt[3];
  gwt_in[0] = df_add(gw[0], df_cross2(u[1], u[2], gv[1], gv[2]));  // d e / d w from v = w x u
  gwt_in[1] = df_add(gw[1], df_cross2(u[2], u[0], gv[2], gv[0]));
  gwt_in[2] = df_add(gw[2], df_cross2(u[0], u[1], gv[0], gv[1]));
  gu[0] = df_cross2(gv[1], gv[2], w[1], w[2]);  // d e / d u from v = w x u
  gu[1] = df_cross2(gv[2], gv[0], w[2], w[0]);
  gu[2] = df_cross2(gv[0], gv[1], w[0], w[1]);
  const df gww = df_dot3(gwt_in, w);
  for (int k = 0; k < 3; ++k) gwt[k] = df_mul(df_sub(gwt_in[k], df_mul(gww, w[k])), inw);
  const df gwu = df_dot3(gwt, u);
  if (ax < 0) {
    for (int k = 0; k < 3; ++k) {
      gup[k] = df_sub(gwt[k], df_mul(gwu, u[k]));
      gu[k] = df_sub(gu[k], df_add(df_mul(gwu, rr[k]), df_mul(ru, gwt[k])));
    }
  } else {
    const df ui = ax == 0 ? u[0] : (ax == 1 ? u[1] : u[2]);
    for (int k = 0; k < 3; ++k) {
      gup[k] = df{0.0f, 0.0f};
      gu[k] = df_sub(gu[k], df_mul(ui, gwt[k]));
    }
    gu[ax] = df_sub(gu[ax], gwu);
  }
  const df guu = df_dot3(gu, u);
  for (int k = 0; k < 3; ++k) {
    const df gd = df_mul(df_sub(gu[k], df_mul(guu, u[k])), ind);
    gCb[k] = gd;
    gCa[k] = df_neg(gd);
  }
  return true;
}

// Valid arc of the pencil for one view: the plane at kappa (c = (cos, sin)) meets
// the detector rectangle iff the values g_c . c at the four corners do not all have
// the same strict sign, g_c = A^T x_c.  If the g_c lie in a half plane (epipole
// outside), the valid directions (mod pi) run counter-clockwise from rot90(g_min)
// over the angle between the extreme g's; otherwise every plane is valid.  The
// corner values, the sign tests (each cross product once, with its antisymmetry for
// the reversed order) and the angle run in double-float.
__host__ __device__ __noinline__ df view_arc(const df* A, int W, int H, df* clo) {
  const float hw = 0.5f * (float)W, hh = 0.5f * (float)H;  // exact
  const float xs[4] = {-hw, hw, hw, -hw};
  const float ys[4] = {-hh, -hh, hh, hh};
  df sc = df_mul(A[0], A[0]);
  for (int k = 1; k < 6; ++k) sc = df_add(sc, df_mul(A[k], A[k]));
  df gx[4], gy[4], n2[4];
  bool degenerate = false;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    gx[c] = df_add(df_add(df_mul_f(A[0], xs[c]), df_mul_f(A[2], ys[c])), A[4]);
    gy[c] = df_add(df_add(df_mul_f(A[1], xs[c]), df_mul_f(A[3], ys[c])), A[5]);
    n2[c] = df_add(df_mul(gx[c], gx[c]), df_mul(gy[c], gy[c]));
    if (!(n2[c].hi > 1e-28f * sc.hi)) degenerate = true;
  }
  // cross products g_i x g_j (i < j); g_j x g_i = -(g_i x g_j)
  const float c01 = df_cross2(gx[0], gy[0], gx[1], gy[1]).hi, c02 = df_cross2(gx[0], gy[0], gx[2], gy[2]).hi;
  const float c03 = df_cross2(gx[0], gy[0], gx[3], gy[3]).hi, c12 = df_cross2(gx[1], gy[1], gx[2], gy[2]).hi;
  const float c13 = df_cross2(gx[1], gy[1], gx[3], gy[3]).hi, c23 = df_cross2(gx[2], gy[2], gx[3], gy[3]).hi;
  // corner i is the minimum if g_i x g_j >= 0 for every j, the maximum if <= 0
  const bool mn0 = c01 >= 0.0f && c02 >= 0.0f && c03 >= 0.0f, mx0 = c01 <= 0.0f && c02 <= 0.0f && c03 <= 0.0f;
  const bool mn1 = -c01 >= 0.0f && c12 >= 0.0f && c13 >= 0.0f, mx1 = -c01 <= 0.0f && c12 <= 0.0f && c13 <= 0.0f;
  const bool mn2 = -c02 >= 0.0f && -c12 >= 0.0f && c23 >= 0.0f, mx2 = -c02 <= 0.0f && -c12 <= 0.0f && c23 <= 0.0f;
  const bool mn3 = -c03 >= 0.0f && -c13 >= 0.0f && -c23 >= 0.0f, mx3 = -c03 <= 0.0f && -c13 <= 0.0f && -c23 <= 0.0f;
  const int imin = mn0 ? 0 : (mn1 ? 1 : (mn2 ? 2 : (mn3 ? 3 : -1)));
  const int imax = mx0 ? 0 : (mx1 ? 1 : (mx2 ? 2 : (mx3 ? 3 : -1)));
  if (degenerate || imin < 0 || imax < 0) {
    clo[0] = df{0.0f, 0.0f};
    clo[1] = df{-1.0f, 0.0f};
    return df_pi();
  }
  // (scalars and selects only: no dynamically indexed local arrays)
  const df ax_ = df_sel(imin == 0, gx[0], df_sel(imin == 1, gx[1], df_sel(imin == 2, gx[2], gx[3])));
  const df ay_ = df_sel(imin == 0, gy[0], df_sel(imin == 1, gy[1], df_sel(imin == 2, gy[2], gy[3])));
  const df an2 = df_sel(imin == 0, n2[0], df_sel(imin == 1, n2[1], df_sel(imin == 2, n2[2], n2[3])));
  const df bx_ = df_sel(imax == 0, gx[0], df_sel(imax == 1, gx[1], df_sel(imax == 2, gx[2], gx[3])));
  const df by_ = df_sel(imax == 0, gy[0], df_sel(imax == 1, gy[1], df_sel(imax == 2, gy[2], gy[3])));
  const df cr = df_cross2(ax_, ay_, bx_, by_);
  const df dt = df_add(df_mul(ax_, bx_), df_mul(ay_, by_));
  df phi = df_atan2(cr, dt);
  if (df_lt0(phi)) phi = df{0.0f, 0.0f};
  const df ing = df_rsqrt(an2);
  clo[0] = df_neg(df_mul(ay_, ing));
  clo[1] = df_mul(ax_, ing);
  return phi;
}

}  // namespace

// Per-pair set-up: frame, kappa -> line maps, valid arcs, the sampled arc, the
// integer ranges of valid samples and the tile-centre directions (ctile, n_tiles
// entries).  With previous != NULL the sampling of *previous is kept and only the maps
// follow the geometry.  GB300 issues FP64 at 1/64 of the FP32 rate, so everything
// here runs in double-float (about 48 bits) on the FP32 pipes from the views'
// double-float copies: the frame, the maps, the corner values and signs, the angles
// (df_atan2, df_sincos), the step and the positions whose floors give the integer
// ranges.
__host__ __device__ PairRec setup_pair(int a, int b, int n_views, const ViewRec* views, int W, int H, int K,
                                       float4* ctile, int n_tiles, const PairRec* previous) {
  const bool reuse_sampling = previous != nullptr;
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
  r.dk_hi = r.dk_lo = 0.0f;
  for (int i = 0; i < 24; ++i) (&r.Af[0][0])[i] = 0.0f;
  r.c0[0] = 1.0;
  r.c0[1] = 0.0;
  const ViewRec& va = views[a];
  const ViewRec& vb = views[b];
  df w[3], v[3];
  df Ad[2][6];
  bool ok = in_range && va.status == 0 && vb.status == 0 && a != b && pencil_frame_df(va, vb, w, v);
  if (ok) {
    const ViewRec* vv[2] = {&va, &vb};
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < 3; ++i) {
        const df row[3] = {qget(*vv[s], 6 + 3 * i), qget(*vv[s], 7 + 3 * i), qget(*vv[s], 8 + 3 * i)};
        Ad[s][2 * i + 0] = df_dot3(row, w);
        Ad[s][2 * i + 1] = df_dot3(row, v);
      }
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < 6; ++i) {
        r.Af[s][2 * i] = Ad[s][i].hi;
        r.Af[s][2 * i + 1] = Ad[s][i].lo;
      }
  }
  if (ok && reuse_sampling) {
    // keep the planes sampled by the previous call (kappa arcs and validity
    // frozen); only the kappa -> line maps follow the new geometry
    const PairRec old = *previous;
    r.dk = old.dk;
    r.c0[0] = old.c0[0];
    r.c0[1] = old.c0[1];
    r.dk_hi = old.dk_hi;
    r.dk_lo = old.dk_lo;
    r.r0lo = old.r0lo;
    r.r0hi = old.r0hi;
    r.r1lo = old.r1lo;
    r.r1hi = old.r1hi;
    r.nk = old.nk;
    ok = old.status == 0;
  } else if (ok) {
    df cla[2], clb[2];
    const df lena = view_arc(Ad[0], W, H, cla);
    const df lenb = view_arc(Ad[1], W, H, clb);
    // sample the shorter arc; ties (equal in exact arithmetic for mirror-symmetric
    // pairs) go to view a within a relative tolerance, not by rounding
    const bool samp_a = df_sub(lena, lenb).hi <= 1e-9f * fmaxf(lena.hi, lenb.hi);
    const df len_s = samp_a ? lena : lenb, len_o = samp_a ? lenb : lena;
    const df csx = samp_a ? cla[0] : clb[0], csy = samp_a ? cla[1] : clb[1];
    const df cox = samp_a ? clb[0] : cla[0], coy = samp_a ? clb[1] : cla[1];
    const df dk = df_div_f(len_s, (float)K);
    r.dk = df_to_double(dk);
    r.dk_hi = dk.hi;
    r.dk_lo = dk.lo;
    // one sincos: the rotations by dk, 16 dk and 32 dk follow by angle doubling (the
    // angle error doubles with each step: about 1e-13 rad after six)
    df sh, ch;
    df_sincos(df_mul_f(dk, 0.5f), &sh, &ch);
    auto twice = [](df& s_, df& c_) {
      const df s2 = df_mul_f(df_mul(s_, c_), 2.0f);
      c_ = df_sub(df_mul(c_, c_), df_mul(s_, s_));
      s_ = s2;
    };
    auto rotate = [](df c, df s, df x, df y, df* ox, df* oy) {
      *ox = df_sub(df_mul(c, x), df_mul(s, y));
      *oy = df_add(df_mul(s, x), df_mul(c, y));
    };
    {
      df c0x, c0y;
      rotate(ch, sh, csx, csy, &c0x, &c0y);
      r.c0[0] = df_to_double(c0x);
      r.c0[1] = df_to_double(c0y);
    }
    // valid samples of the other view: y_k = delta0 + (k + 1/2) dk, valid iff
    // y_k <= len_o or pi <= y_k <= pi + len_o (angles mod pi from its arc start)
    const df pi = df_pi();
    if (!df_lt0(df_sub(len_o, pi))) {
      r.r0lo = 0;
      r.r0hi = K;
      r.r1lo = r.r1hi = K;
    } else if (dk.hi > 0.0f) {
      df d0 = df_atan2(df_cross2(cox, coy, csx, csy), df_add(df_mul(cox, csx), df_mul(coy, csy)));
      if (df_lt0(d0)) d0 = df_add(d0, pi);
      if (!df_lt0(df_sub(d0, pi))) d0 = df_sub(d0, pi);
      const df idk = df_recip(dk);
      const df half = {0.5f, 0.0f};
      // floor / ceil of the sample positions (integer-valued FP32; K is exact in FP32)
      float fr;
      const float e0 = df_floor_frac(df_sub(df_mul(df_sub(len_o, d0), idk), half), &fr);
      float s1 = df_floor_frac(df_sub(df_mul(df_sub(pi, d0), idk), half), &fr);
      if (fr > 0.0f) s1 += 1.0f;
      const float e1 = df_floor_frac(df_sub(df_mul(df_sub(df_add(pi, len_o), d0), idk), half), &fr);
      const float Kf = (float)K;
      const int hi0 = (int)fminf(fmaxf(e0 + 1.0f, 0.0f), Kf);
      const int lo1 = (int)fminf(fmaxf(s1, (float)hi0), Kf);
      const int hi1 = (int)fminf(fmaxf(e1 + 1.0f, (float)lo1), Kf);
      r.r0lo = 0;
      r.r0hi = hi0;
      r.r1lo = lo1;
      r.r1hi = hi1;
    }
    r.nk = (r.r0hi - r.r0lo) + (r.r1hi - r.r1lo);
    // directions of the tile centres: tile t holds samples [32t, min(32t + 32, K)),
    // centred at ((k_begin + k_end) / 2) dk from the arc start; full tiles step by 32 dk
    df s16 = sh, c16 = ch;
    for (int i = 0; i < 5; ++i) twice(s16, c16);  // 16 dk
    df s32 = s16, c32 = c16;
    twice(s32, c32);  // 32 dk
    df cx0, cy0;
    rotate(c16, s16, csx, csy, &cx0, &cy0);
    float4* ct = ctile;
    for (int t = 0; t < n_tiles; ++t) {
      if (32 * t + 32 <= K) {
        ct[t] = make_float4(cx0.hi, cy0.hi, cx0.lo, cy0.lo);
      } else {  // last, partial tile
        df sp, cp, px, py;
        df_sincos(df_mul_f(dk, 0.5f * (float)(32 * t + K)), &sp, &cp);
        rotate(cp, sp, csx, csy, &px, &py);
        ct[t] = make_float4(px.hi, py.hi, px.lo, py.lo);
      }
      df nx, ny;
      rotate(c32, s32, cx0, cy0, &nx, &ny);
      cx0 = nx;
      cy0 = ny;
    }
  }
  if (!ok) r.status = 1;
  return r;
}

__global__ void pair_setup_kernel(int n_views, long long p_begin, long long p_end, const int32_t* __restrict__ pairs,
                                  const ViewRec* __restrict__ views, int W, int H, int K,
                                  PairRec* __restrict__ out, float4* __restrict__ ctile, int n_tiles,
                                  int reuse_sampling, int* __restrict__ status) {
  const long long p = p_begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= p_end) return;
  int a, b;
  if (pairs) {
    a = pairs[2 * p];
    b = pairs[2 * p + 1];
  } else {
    pair_from_index(p, n_views, &a, &b);
  }
  PairRec prev;
  if (reuse_sampling) prev = out[p];
  const PairRec r = setup_pair(a, b, n_views, views, W, H, K, ctile + p * n_tiles, n_tiles,
                               reuse_sampling ? &prev : nullptr);
  if (r.status) atomicOr(status, kStatusDegeneratePair);
  out[p] = r;
}

// Gradient of one pair's e with respect to the per-view quantities the pair reads,
// q = (C[3], up[3], cofc[9]) of view a, then of view b (30 values), from
// G = d e / d A (the pair kernel's adjoint, FP32 values): A = cofc [w v] is linear in
// cofc, and the frame (w, v) is differentiated in reverse mode
// (pencil_frame_adjoint_df).  Double-float throughout; out holds (hi, lo) pairs.
__device__ void pair_grad_q(const PairRec& pr, const ViewRec* __restrict__ views, const double* __restrict__ G,
                            float2* __restrict__ out) {
  if (pr.status != 0 || pr.nk <= 0) {
    for (int j = 0; j < 30; ++j) out[j] = make_float2(0.0f, 0.0f);
    return;
  }
  const ViewRec& va = views[pr.a];
  const ViewRec& vb = views[pr.b];
  const ViewRec* vv[2] = {&va, &vb};
  df g[12];
  for (int i = 0; i < 12; ++i) g[i] = df{(float)G[i], 0.0f};  // an FP32 value: exact
  // d e / d w and d e / d v through A = cofc [w v]
  df gw[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}}, gv[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 3; ++i) {
      const df g0 = g[6 * s + 2 * i], g1 = g[6 * s + 2 * i + 1];
      for (int k = 0; k < 3; ++k) {
        const df cof = qget(*vv[s], 6 + 3 * i + k);
        gw[k] = df_add(gw[k], df_mul(g0, cof));
        gv[k] = df_add(gv[k], df_mul(g1, cof));
      }
    }
  df w[3], v[3], gCa[3], gCb[3], gup[3];
  if (!pencil_frame_adjoint_df(va, vb, gw, gv, w, v, gCa, gCb, gup)) {
    for (int j = 0; j < 30; ++j) out[j] = make_float2(0.0f, 0.0f);
    return;
  }
  auto put = [&](int j, df x) { out[j] = make_float2(x.hi, x.lo); };
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 3; ++i) {
      const df g0 = g[6 * s + 2 * i], g1 = g[6 * s + 2 * i + 1];
      for (int k = 0; k < 3; ++k) put(15 * s + 6 + 3 * i + k, df_add(df_mul(g0, w[k]), df_mul(g1, v[k])));
    }
  for (int k = 0; k < 3; ++k) {
    put(k, gCa[k]);
    put(3 + k, gup[k]);
    put(15 + k, gCb[k]);
    put(18 + k, gup[k]);
  }
}

__global__ void pair_grad_q_kernel(long long n_pairs, const PairRec* __restrict__ prs,
                                   const ViewRec* __restrict__ views, const double* __restrict__ Gpp,
                                   float2* __restrict__ gq) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pairs) return;
  pair_grad_q(prs[p], views, Gpp + 12 * p, gq + 30 * p);
}

// Per-view sum of the pairs' q gradients in a fixed order (one block of 256 threads
// per view), in double-float: on return sh[k][0] (k < 15) holds d total / d q_k of view
// lam as a (hi, lo) pair.  With pairs == NULL the pairs of a view are found by the
// row-major a < b enumeration, otherwise by scanning the pair list.
__device__ void reduce_q_block(int lam, int n_views, long long n_pairs, const int32_t* __restrict__ pairs,
                               const float2* __restrict__ gq, float2 (*sh)[256]) {
  df acc[15];
  for (int k = 0; k < 15; ++k) acc[k] = df{0.0f, 0.0f};
  auto add = [&](const float2* q) {
    for (int k = 0; k < 15; ++k) {
      const float2 x = q[k];
      acc[k] = df_add(acc[k], df{x.x, x.y});
    }
  };
  if (pairs) {
    for (long long p = threadIdx.x; p < n_pairs; p += blockDim.x) {
      const int a = pairs[2 * p], b = pairs[2 * p + 1];
      if (a == lam) add(gq + 30 * p);
      if (b == lam) add(gq + 30 * p + 15);
    }
  } else {
    const long long n = n_views;
    for (int o = threadIdx.x; o < n_views; o += blockDim.x) {
      if (o == lam) continue;
      const long long a = o < lam ? o : lam, b = o < lam ? lam : o;
      const long long p = a * (2 * n - a - 1) / 2 + (b - a - 1);
      const int off = o < lam ? 15 : 0;  // this view is b of the pair when o < lam
      add(gq + 30 * p + off);
    }
  }
  for (int k = 0; k < 15; ++k) sh[k][threadIdx.x] = make_float2(acc[k].hi, acc[k].lo);
  __syncthreads();
  for (int wdt = blockDim.x / 2; wdt > 0; wdt >>= 1) {
    if (threadIdx.x < wdt)
      for (int k = 0; k < 15; ++k) {
        const float2 x = sh[k][threadIdx.x], y = sh[k][threadIdx.x + wdt];
        const df z = df_add(df{x.x, x.y}, df{y.x, y.y});
        sh[k][threadIdx.x] = make_float2(z.hi, z.lo);
      }
    __syncthreads();
  }
}

__device__ __forceinline__ double sh_value(const float2 (*sh)[256], int k) {
  return (double)sh[k][0].x + (double)sh[k][0].y;
}

// d total / d theta of one view from its q gradient (sh[k][0]) and the tangents
// d q / d theta (C, up, cofc rows).
__device__ __forceinline__ double contract_theta(const float2 (*sh)[256], const ViewTan& t, int j) {
  double g = 0.0;
  for (int k = 0; k < 3; ++k) g += sh_value(sh, k) * t.dC[k][j];
  for (int k = 0; k < 3; ++k) g += sh_value(sh, 3 + k) * t.dup[k][j];
  for (int k = 0; k < 9; ++k) g += sh_value(sh, 6 + k) * t.dcofc[k][j];
  return g;
}

// grad[view][6] = d total / d theta (one block of 256 threads per view).
__global__ void __launch_bounds__(256) view_grad_theta_kernel(int n_views, long long n_pairs,
                                                              const int32_t* __restrict__ pairs,
                                                              const float2* __restrict__ gq,
                                                              const ViewTan* __restrict__ vtan,
                                                              double* __restrict__ grad) {
  __shared__ float2 sh[15][256];
  const int lam = blockIdx.x;
  reduce_q_block(lam, n_views, n_pairs, pairs, gq, sh);
  if (threadIdx.x < 6) grad[6 * lam + threadIdx.x] = contract_theta(sh, vtan[lam], threadIdx.x);
}

// grad_P[view][12] = d total / d P (one block of 256 threads per view).
__global__ void __launch_bounds__(256) view_grad_P_kernel(int n_views, long long n_pairs,
                                                          const int32_t* __restrict__ pairs,
                                                          const float2* __restrict__ gq,
                                                          const ViewTanP* __restrict__ vtan,
                                                          double* __restrict__ grad_P) {
  __shared__ float2 sh[15][256];
  const int lam = blockIdx.x;
  reduce_q_block(lam, n_views, n_pairs, pairs, gq, sh);
  if (threadIdx.x < 12) {
    const ViewTanP& t = vtan[lam];
    double g = 0.0;
    for (int k = 0; k < 15; ++k) g += sh_value(sh, k) * t.d[k][threadIdx.x];
    grad_P[12 * lam + threadIdx.x] = g;
  }
}

// ---------------------------------------------------------------- serving rounds
__global__ void serve_view_kernel(const ServeJob* __restrict__ jobs, const long long* __restrict__ voff, int n_jobs,
                                  long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int j = serve_job_of(voff, n_jobs, i);
  const ServeJob& J = jobs[j];
  const long long v = i - voff[j];
  const ViewRec r = setup_view(J.P + 12 * v, J.theta + 6 * v, J.W, J.H);
  if (r.status) atomicOr(J.status, kStatusDegenerateView);
  J.views[v] = r;
  if (J.do_grad) J.vtan[v] = view_tangent(J.P + 12 * v, J.theta + 6 * v, J.W, J.H);
}

__global__ void serve_pair_setup_kernel(const ServeJob* __restrict__ jobs, const long long* __restrict__ poff,
                                        int n_jobs, long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int j = serve_job_of(poff, n_jobs, i);
  const ServeJob& J = jobs[j];
  const long long p = i - poff[j];
  int a, b;
  pair_from_index(p, J.n_views, &a, &b);
  const PairRec r = setup_pair(a, b, J.n_views, J.views, J.W, J.H, J.pair.K,
                               const_cast<float4*>(J.pair.ctile) + p * J.n_tiles, J.n_tiles, nullptr);
  if (r.status) atomicOr(J.status, kStatusDegeneratePair);
  const_cast<PairRec*>(J.pair.prs)[p] = r;
}

__global__ void serve_pair_grad_kernel(const ServeJob* __restrict__ jobs, const long long* __restrict__ poff,
                                       int n_jobs, long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int j = serve_job_of(poff, n_jobs, i);
  const ServeJob& J = jobs[j];
  if (!J.do_grad) return;
  const long long p = i - poff[j];
  pair_grad_q(J.pair.prs[p], J.views, J.pair.Gpp + 12 * p, J.gpp + 30 * p);
}

__global__ void __launch_bounds__(256) serve_view_grad_kernel(const ServeJob* __restrict__ jobs,
                                                              const long long* __restrict__ voff, int n_jobs) {
  __shared__ float2 sh[15][256];
  const long long i = blockIdx.x;
  const int j = serve_job_of(voff, n_jobs, i);
  const ServeJob& J = jobs[j];
  if (!J.do_grad) return;  // block-uniform
  const int lam = (int)(i - voff[j]);
  reduce_q_block(lam, J.n_views, J.pair.n_pairs, nullptr, J.gpp, sh);
  if (threadIdx.x < 6) J.grad[6 * lam + threadIdx.x] = contract_theta(sh, J.vtan[lam], threadIdx.x);
}

// Per-view jobs: theta <- theta - step * grad for the estimated parameters.
__global__ void serve_step_kernel(const ServeJob* __restrict__ jobs, const long long* __restrict__ voff, int n_jobs,
                                  long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * total) return;
  const int j = serve_job_of(voff, n_jobs, i / 6);
  const ServeJob& J = jobs[j];
  const long long k = i - 6 * voff[j];
  if (!J.do_grad || J.model != kMotionPerView || !(J.mask >> (int)(k % 6) & 1)) return;
  J.theta[k] = J.theta[k] - J.step * J.grad[k];
}

// Spline jobs: theta = theta0 + Akima(nodes) for the estimated parameters, and the
// window Jacobian of each (view, parameter).
__global__ void serve_spline_kernel(const ServeJob* __restrict__ jobs, const long long* __restrict__ voff,
                                    int n_jobs, long long total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 6 * total) return;
  const int j = serve_job_of(voff, n_jobs, i / 6);
  const ServeJob& J = jobs[j];
  if (J.model != kMotionAkima) return;
  const long long k = i - 6 * voff[j];
  const int p = (int)(k % 6);
  const long long v = k / 6;
  if (!(J.mask >> p & 1)) {
    J.theta[k] = J.theta0[k];
    return;
  }
  const AkimaPoint a = akima_point(J.nodes + p, 6, J.n_nodes, J.h, (double)v);
  J.theta[k] = J.theta0[k] + a.value;
  for (int q = 0; q < 6; ++q) J.jac[6 * k + q] = a.d[q];
  J.jbase[k] = a.base;
}

// Spline jobs: node gradient d total / d y_(n, p) = sum over the views whose window
// holds node n of jac * grad, summed in view order; then the step on the nodes.
// One thread per (node, parameter) of a job, one block per job.
__global__ void serve_node_step_kernel(const ServeJob* __restrict__ jobs) {
  const ServeJob& J = jobs[blockIdx.x];
  if (!J.do_grad || J.model != kMotionAkima) return;
  for (int t = threadIdx.x; t < 6 * J.n_nodes; t += blockDim.x) {
    const int node = t / 6, p = t % 6;
    if (!(J.mask >> p & 1)) continue;
    // windows [i - 2, i + 3] hold node n for intervals i in [n - 3, n + 2]: views in
    // [(n - 3) h, (n + 3) h]
    const long long v0 = (long long)fmax(0.0, floor((node - 3) * J.h));
    const long long v1 = (long long)fmin((double)(J.n_views - 1), ceil((node + 3) * J.h));
    double g = 0.0;
    for (long long v = v0; v <= v1; ++v) {
      const long long k = 6 * v + p;
      const int q = node - J.jbase[k];
      if (q >= 0 && q < 6) g += J.jac[6 * k + q] * J.grad[k];
    }
    J.nodes[t] = J.nodes[t] - J.step * g;
  }
}

cudaError_t launch_serve_motion(const ServeJob* jobs, const long long* voff, int n_jobs, long long n_views,
                                cudaStream_t stream) {
  if (n_views > 0)
    serve_spline_kernel<<<(unsigned)((6 * n_views + 127) / 128), 128, 0, stream>>>(jobs, voff, n_jobs, n_views);
  return cudaGetLastError();
}

cudaError_t launch_serve_setup(const ServeJob* jobs, const long long* voff, const long long* poff, int n_jobs,
                               long long n_views, long long n_pairs, cudaStream_t stream) {
  if (n_views > 0) serve_view_kernel<<<(unsigned)((n_views + 63) / 64), 64, 0, stream>>>(jobs, voff, n_jobs, n_views);
  if (n_pairs > 0)
    serve_pair_setup_kernel<<<(unsigned)((n_pairs + 127) / 128), 128, 0, stream>>>(jobs, poff, n_jobs, n_pairs);
  return cudaGetLastError();
}

cudaError_t launch_serve_grad(const ServeJob* jobs, const long long* voff, const long long* poff, int n_jobs,
                              long long n_views, long long n_pairs, cudaStream_t stream) {
  if (n_pairs > 0)
    serve_pair_grad_kernel<<<(unsigned)((n_pairs + 63) / 64), 64, 0, stream>>>(jobs, poff, n_jobs, n_pairs);
  if (n_views > 0) {
    serve_view_grad_kernel<<<(unsigned)n_views, 256, 0, stream>>>(jobs, voff, n_jobs);
    serve_step_kernel<<<(unsigned)((6 * n_views + 255) / 256), 256, 0, stream>>>(jobs, voff, n_jobs, n_views);
    serve_node_step_kernel<<<n_jobs, 128, 0, stream>>>(jobs);
  }
  return cudaGetLastError();
}

__global__ void alpha_dir_kernel(int n_alpha, float4* __restrict__ dir) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_alpha) return;
  double s, c;
  sincospi((double)m / (double)n_alpha, &s, &c);
  dir[m] = split_dir(c, s);
}

}  // namespace ecc

// Internal host entry point (tests only, not part of the public ABI): runs the
// per-view and per-pair set-up above on the CPU for views (a, b) of a scan so
// that the set-up logic can be checked without a GPU.
//   P host FP64 [n_views][12], motion host FP64 [n_views][6] or NULL
//   info_out [8]: sampled-arc start direction of sample 0 (c0x, c0y), dk, nk,
//                 status, r0hi, r1lo, r1hi
//   A_out [12]: the kappa -> line maps of views a and b
extern "C" int ecc_internal_setup_pair_host(int n_views, const double* P, const double* motion, int W, int H, int K,
                                            int a, int b, double* info_out, double* A_out) {
  if (n_views < 1 || a < 0 || b < 0 || a >= n_views || b >= n_views || K < 1) return -1;
  ecc::ViewRec views[2];
  views[0] = ecc::setup_view(P + 12 * a, motion ? motion + 6 * a : nullptr, W, H);
  views[1] = ecc::setup_view(P + 12 * b, motion ? motion + 6 * b : nullptr, W, H);
  const int n_tiles = (K + 31) / 32;
  float4* ct = new float4[n_tiles];
  const ecc::PairRec r = ecc::setup_pair(0, 1, 2, views, W, H, K, ct, n_tiles, nullptr);
  delete[] ct;
  info_out[0] = r.c0[0];
  info_out[1] = r.c0[1];
  info_out[2] = r.dk;
  info_out[3] = r.nk;
  info_out[4] = r.status;
  info_out[5] = r.r0hi;
  info_out[6] = r.r1lo;
  info_out[7] = r.r1hi;
  for (int i = 0; i < 12; ++i) A_out[i] = (double)(&r.Af[0][0])[2 * i] + (double)(&r.Af[0][0])[2 * i + 1];
  return 0;
}

// Internal host entry point (tests only): the Akima spline point of the motion
// model, computed by the same code as the serving kernels.
//   y host FP64 [n] node values, h node spacing, x position; out[0] value, out[1..6]
//   derivatives with respect to y[base .. base + 5]; *base receives base.
extern "C" int ecc_internal_akima_host(const double* y, int n, double h, double x, double* out, int* base) {
  if (!y || !out || !base || n < 3 || !(h > 0.0)) return -1;
  const ecc::AkimaPoint a = ecc::akima_point(y, 1, n, h, x);
  out[0] = a.value;
  for (int k = 0; k < 6; ++k) out[1 + k] = a.d[k];
  *base = a.base;
  return 0;
}

// Internal host entry point (tests only): the double-float angle functions of the
// per-pair set-up on the CPU.  op 0: out[2i], out[2i + 1] = sin, cos of x[i] (|x| <= 4);
// op 1: out[i] = atan2(x[i], y[i]).  Inputs are split into double-float pairs first.
extern "C" int ecc_internal_df_math_host(int op, const double* x, const double* y, int n, double* out) {
  if (!x || !out || n < 0 || (op == 1 && !y) || op < 0 || op > 1) return -1;
  for (int i = 0; i < n; ++i) {
    if (op == 0) {
      ecc::df s, c;
      ecc::df_sincos(ecc::df_from_double(x[i]), &s, &c);
      out[2 * i] = ecc::df_to_double(s);
      out[2 * i + 1] = ecc::df_to_double(c);
    } else {
      out[i] = ecc::df_to_double(ecc::df_atan2(ecc::df_from_double(x[i]), ecc::df_from_double(y[i])));
    }
  }
  return 0;
}

// Internal host entry point (tests only): the pencil frame of two sources and its
// reverse mode (pencil_frame_df, pencil_frame_adjoint_df) on the CPU.
//   Ca, Cb, upa, upb [3] host FP64; gw, gv [3] the incoming d e / d w, d e / d v
//   w_v_out [6] = w, v; grad_out [9] = d e / d Ca, d e / d Cb, d e / d up (each up axis)
// Returns -1 for coincident sources.
extern "C" int ecc_internal_frame_adjoint_host(const double* Ca, const double* Cb, const double* upa,
                                               const double* upb, const double* gw, const double* gv,
                                               double* w_v_out, double* grad_out) {
  ecc::ViewRec va{}, vb{};
  for (int k = 0; k < 3; ++k) {
    const ecc::df ca = ecc::df_from_double(Ca[k]), cb = ecc::df_from_double(Cb[k]);
    const ecc::df ua = ecc::df_from_double(upa[k]), ub = ecc::df_from_double(upb[k]);
    va.qdf[2 * k] = ca.hi; va.qdf[2 * k + 1] = ca.lo;
    vb.qdf[2 * k] = cb.hi; vb.qdf[2 * k + 1] = cb.lo;
    va.qdf[6 + 2 * k] = ua.hi; va.qdf[6 + 2 * k + 1] = ua.lo;
    vb.qdf[6 + 2 * k] = ub.hi; vb.qdf[6 + 2 * k + 1] = ub.lo;
  }
  ecc::df g_w[3], g_v[3], w[3], v[3], gCa[3], gCb[3], gup[3];
  for (int k = 0; k < 3; ++k) {
    g_w[k] = ecc::df_from_double(gw[k]);
    g_v[k] = ecc::df_from_double(gv[k]);
  }
  if (!ecc::pencil_frame_adjoint_df(va, vb, g_w, g_v, w, v, gCa, gCb, gup)) return -1;
  for (int k = 0; k < 3; ++k) {
    w_v_out[k] = ecc::df_to_double(w[k]);
    w_v_out[3 + k] = ecc::df_to_double(v[k]);
    grad_out[k] = ecc::df_to_double(gCa[k]);
    grad_out[3 + k] = ecc::df_to_double(gCb[k]);
    grad_out[6 + k] = ecc::df_to_double(gup[k]);
  }
  return 0;
}
