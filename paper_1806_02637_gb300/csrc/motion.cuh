// Spline motion model: each rigid motion parameter of the trajectory as an Akima
// spline over the view index (Optimization section; Akima 1970), nodes uniform at
// x_j = j h, h = (n_views - 1) / (n_nodes - 1).  A point on interval i depends on
// the node values y_(i-2) .. y_(i+3); akima_point returns the value and, by
// forward-mode dual numbers (FP64), its derivatives with respect to those six.
#pragma once
#include <cuda_runtime.h>

#include "dual.cuh"

namespace ecc {

enum : int { kMotionPerView = 0, kMotionAkima = 1 };

struct AkimaPoint {
  double value;
  double d[6];  // d value / d y_(base + k)
  int base;     // i - 2
};

namespace akima_detail {

using D6 = Dual<6>;

__host__ __device__ inline D6 dabs(const D6& a) { return a.v < 0.0 ? -a : a; }

// Interval slope m_k (k = -2 .. n of Akima's extended sequence) from the local
// node values yl[j - base], j = base .. base + 5.
__host__ __device__ inline D6 slope(const D6* yl, int base, int n, double h, int k) {
  const double ih = 1.0 / h;
  auto m_in = [&](int j) { return (yl[j + 1 - base] - yl[j - base]) * ih; };  // 0 <= j <= n - 2
  if (k >= 0 && k <= n - 2) return m_in(k);
  if (k == -1) return 2.0 * m_in(0) - m_in(1);
  if (k == -2) return 3.0 * m_in(0) - 2.0 * m_in(1);  // 2 m_(-1) - m_0
  if (k == n - 1) return 2.0 * m_in(n - 2) - m_in(n - 3);
  return 3.0 * m_in(n - 2) - 2.0 * m_in(n - 3);      // k == n: 2 m_(n-1) - m_(n-2)
}

// Node derivative t_j from m_(j-2) .. m_(j+1).
__host__ __device__ inline D6 node_slope(const D6* yl, int base, int n, double h, int j) {
  const D6 mm2 = slope(yl, base, n, h, j - 2), mm1 = slope(yl, base, n, h, j - 1);
  const D6 m0 = slope(yl, base, n, h, j), mp1 = slope(yl, base, n, h, j + 1);
  const D6 w1 = dabs(mp1 - m0), w2 = dabs(mm1 - mm2);
  const D6 ws = w1 + w2;
  if (ws.v == 0.0) return 0.5 * (mm1 + m0);
  return (w1 * mm1 + w2 * m0) / ws;
}

}  // namespace akima_detail

// Value at x (0 <= x <= n_views - 1) of the Akima spline through the node values
// y[0], y[stride], ..., y[(n - 1) stride] (n >= 3), and its node derivatives.
__host__ __device__ inline AkimaPoint akima_point(const double* y, int stride, int n, double h, double x) {
  using namespace akima_detail;
  int i = (int)floor(x / h);
  i = i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
  const int base = i - 2;
  D6 yl[6];
  for (int k = 0; k < 6; ++k) {
    const int j = base + k;
    yl[k] = D6(j >= 0 && j < n ? y[(long long)j * stride] : 0.0);
    yl[k].d[k] = j >= 0 && j < n ? 1.0 : 0.0;
  }
  const D6 ti = node_slope(yl, base, n, h, i), ti1 = node_slope(yl, base, n, h, i + 1);
  const double u = (x - i * h) / h;
  const double h00 = (1.0 + 2.0 * u) * (1.0 - u) * (1.0 - u), h10 = u * (1.0 - u) * (1.0 - u);
  const double h01 = u * u * (3.0 - 2.0 * u), h11 = u * u * (u - 1.0);
  const D6 v = h00 * yl[2] + (h10 * h) * ti + h01 * yl[3] + (h11 * h) * ti1;
  AkimaPoint p;
  p.value = v.v;
  for (int k = 0; k < 6; ++k) p.d[k] = v.d[k];
  p.base = base;
  return p;
}

}  // namespace ecc
