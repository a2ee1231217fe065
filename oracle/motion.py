"""Oracle of the spline motion model (test infrastructure: only tests/, the smoke
check and the bench's CPU baseline use this package).

The paper models each rigid motion parameter of the trajectory by an Akima spline
over the projections, so that the optimiser searches only the spline nodes
(Optimization section; H. Akima, "A new method of interpolation and smooth curve
fitting based on local procedures", J. ACM 17, 1970).  Nodes are uniform over the
view index: x_j = j (n_views - 1) / (n_nodes - 1), j = 0 .. n_nodes - 1.

Akima's construction, written out plainly (FP64, numpy):
  * interval slopes m_j = (y_(j+1) - y_j) / (x_(j+1) - x_j), j = 0 .. n - 2;
  * two more slopes at each end by linear extrapolation of the slopes:
      m_(-1) = 2 m_0 - m_1,  m_(-2) = 2 m_(-1) - m_0,
      m_(n-1) = 2 m_(n-2) - m_(n-3),  m_n = 2 m_(n-1) - m_(n-2);
  * node derivative t_j = (|m_(j+1) - m_j| m_(j-1) + |m_(j-1) - m_(j-2)| m_j)
                          / (|m_(j+1) - m_j| + |m_(j-1) - m_(j-2)|),
    and (m_(j-1) + m_j) / 2 where both weights vanish;
  * cubic Hermite interpolation on each interval with values y and derivatives t.

The Jacobian d theta(x) / d y_j is taken by central differences (the construction
is piecewise smooth in the node values: |.| has kinks where two slopes are equal);
tests use node values away from those kinks.
"""
from __future__ import annotations

import numpy as np


def node_positions(n_views: int, n_nodes: int) -> np.ndarray:
    return np.arange(n_nodes, dtype=np.float64) * ((n_views - 1) / (n_nodes - 1))


def akima_slopes(x, y):
    """Node derivatives t_j of Akima's spline through (x_j, y_j)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = len(x)
    if n < 3:
        raise ValueError("Akima's construction needs at least 3 nodes")
    m = np.empty(n + 3)                       # m[k + 2] = m_k, k = -2 .. n
    m[2:n + 1] = np.diff(y) / np.diff(x)      # m_0 .. m_(n-2)
    m[1] = 2.0 * m[2] - m[3]                  # m_(-1)
    m[0] = 2.0 * m[1] - m[2]                  # m_(-2)
    m[n + 1] = 2.0 * m[n] - m[n - 1]          # m_(n-1)
    m[n + 2] = 2.0 * m[n + 1] - m[n]          # m_n
    t = np.empty(n)
    for j in range(n):
        mm2, mm1, m0, mp1 = m[j], m[j + 1], m[j + 2], m[j + 3]   # m_(j-2), m_(j-1), m_j, m_(j+1)
        w1, w2 = abs(mp1 - m0), abs(mm1 - mm2)
        t[j] = 0.5 * (mm1 + m0) if w1 + w2 == 0.0 else (w1 * mm1 + w2 * m0) / (w1 + w2)
    return t


def akima_eval(x, y, xq):
    """Akima spline through (x, y) evaluated at the points xq (inside [x_0, x_(n-1)])."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    xq = np.atleast_1d(np.asarray(xq, dtype=np.float64))
    t = akima_slopes(x, y)
    out = np.empty(len(xq))
    for q, xv in enumerate(xq):
        i = int(np.clip(np.searchsorted(x, xv, side="right") - 1, 0, len(x) - 2))
        h = x[i + 1] - x[i]
        u = (xv - x[i]) / h
        h00 = (1 + 2 * u) * (1 - u) ** 2
        h10 = u * (1 - u) ** 2
        h01 = u * u * (3 - 2 * u)
        h11 = u * u * (u - 1)
        out[q] = h00 * y[i] + h10 * h * t[i] + h01 * y[i + 1] + h11 * h * t[i + 1]
    return out


def akima_jacobian(x, y, xq, step: float = 1e-6):
    """d akima_eval(x, y, xq) / d y, shape [len(xq), len(y)], by central differences."""
    y = np.asarray(y, dtype=np.float64)
    J = np.empty((len(np.atleast_1d(xq)), len(y)))
    for j in range(len(y)):
        yp, ym = y.copy(), y.copy()
        yp[j] += step
        ym[j] -= step
        J[:, j] = (akima_eval(x, yp, xq) - akima_eval(x, ym, xq)) / (2 * step)
    return J


def spline_motion(n_views: int, nodes, motion0=None, param_mask: int = 0x3F):
    """Per-view motion theta [n_views, 6]: motion0 plus, for the parameters whose bit
    is set in param_mask, the Akima spline of nodes [n_nodes, 6] over the view index."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = node_positions(n_views, nodes.shape[0])
    th = np.zeros((n_views, 6)) if motion0 is None else np.array(motion0, dtype=np.float64)
    lam = np.arange(n_views, dtype=np.float64)
    for p in range(6):
        if param_mask >> p & 1:
            th[:, p] += akima_eval(x, nodes[:, p], lam)
    return th


def node_gradient(n_views: int, nodes, grad_theta, param_mask: int = 0x3F):
    """Chain rule: d total / d nodes = J^T d total / d theta per masked parameter."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = node_positions(n_views, nodes.shape[0])
    lam = np.arange(n_views, dtype=np.float64)
    g = np.zeros_like(nodes)
    for p in range(6):
        if param_mask >> p & 1:
            g[:, p] = akima_jacobian(x, nodes[:, p], lam).T @ np.asarray(grad_theta)[:, p]
    return g
