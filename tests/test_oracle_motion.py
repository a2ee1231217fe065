"""Pins of the oracle's Akima spline motion model (CPU, no GPU).

* the spline equals SciPy's Akima1DInterpolator (an independent implementation of
  Akima 1970, same end extrapolation) on random data;
* it interpolates its nodes and reproduces straight lines exactly;
* the Jacobian with respect to the node values: rows sum to one (a constant shift of
  the nodes shifts the spline), J y = f(y) (the construction is positively
  homogeneous of degree one in y, Euler's theorem), and a point depends on six nodes
  at most (locality of Akima's slopes)."""
import numpy as np
import pytest

from oracle import motion as mo

scipy_interp = pytest.importorskip("scipy.interpolate")


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = mo.node_positions(496, n)
    y = rng.normal(0.0, 2.0, n)
    return x, y


@pytest.mark.parametrize("n,seed", [(3, 1), (5, 2), (17, 3), (17, 4), (40, 5)])
def test_akima_matches_scipy(n, seed):
    x, y = _data(n, seed)
    xq = np.linspace(x[0], x[-1], 997)
    ref = scipy_interp.Akima1DInterpolator(x, y)(xq)
    got = mo.akima_eval(x, y, xq)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(y))


def test_nodes_and_lines_reproduced():
    x, y = _data(17, 7)
    assert np.allclose(mo.akima_eval(x, y, x), y, rtol=0, atol=1e-13)
    line = 0.3 - 0.02 * x
    xq = np.linspace(x[0], x[-1], 301)
    assert np.allclose(mo.akima_eval(x, line, xq), 0.3 - 0.02 * xq, rtol=0, atol=1e-12)


def test_jacobian_properties():
    x, y = _data(17, 8)
    xq = np.linspace(x[0], x[-1], 123)
    J = mo.akima_jacobian(x, y, xq)
    assert np.allclose(J.sum(axis=1), 1.0, atol=1e-7)
    assert np.allclose(J @ y, mo.akima_eval(x, y, xq), atol=1e-6 * np.max(np.abs(y)))
    for q, xv in enumerate(xq):
        i = int(np.clip(np.searchsorted(x, xv, side="right") - 1, 0, len(x) - 2))
        outside = [j for j in range(len(x)) if j < i - 2 or j > i + 3]
        assert np.all(J[q, outside] == 0.0)


def test_spline_motion_and_node_gradient():
    rng = np.random.default_rng(9)
    nodes = rng.normal(0.0, 1.0, (17, 6))
    base = rng.normal(0.0, 0.1, (50, 6))
    th = mo.spline_motion(50, nodes, base, param_mask=0b100100)
    assert np.array_equal(th[:, [0, 1, 3, 4]], base[:, [0, 1, 3, 4]])
    x = mo.node_positions(50, 17)
    assert np.allclose(th[:, 5] - base[:, 5], mo.akima_eval(x, nodes[:, 5], np.arange(50)))
    g = rng.normal(0.0, 1.0, (50, 6))
    gn = mo.node_gradient(50, nodes, g, param_mask=0b100000)
    J = mo.akima_jacobian(x, nodes[:, 5], np.arange(50))
    assert np.allclose(gn[:, 5], J.T @ g[:, 5])
    assert np.all(gn[:, :5] == 0.0)
