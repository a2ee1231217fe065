"""The library's Akima motion-model code (run on the CPU through an internal host
entry point) against the oracle's spline: values and the six-node Jacobian window."""
import ctypes

import numpy as np
import pytest

from oracle import motion as mo
from paper_1806_02637_gb300 import build as ecc_build

_dp = ctypes.POINTER(ctypes.c_double)


def _point(y, h, x):
    lib = ctypes.CDLL(ecc_build.build())
    f = lib.ecc_internal_akima_host
    f.argtypes = [_dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, ctypes.POINTER(ctypes.c_int)]
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(7)
    base = ctypes.c_int(0)
    assert f(y.ctypes.data_as(_dp), len(y), h, x, out.ctypes.data_as(_dp), ctypes.byref(base)) == 0
    return out[0], out[1:], base.value


@pytest.mark.parametrize("n_nodes,n_views,seed", [(17, 496, 1), (3, 20, 2), (4, 9, 3), (9, 248, 4)])
def test_library_akima_matches_oracle(n_nodes, n_views, seed):
    rng = np.random.default_rng(seed)
    y = rng.normal(0.0, 2.0, n_nodes)
    xn = mo.node_positions(n_views, n_nodes)
    h = xn[1] - xn[0]
    lam = np.arange(n_views, dtype=np.float64)
    ref = mo.akima_eval(xn, y, lam)
    J = mo.akima_jacobian(xn, y, lam)
    for q, x in enumerate(lam):
        v, d, base = _point(y, h, x)
        assert abs(v - ref[q]) <= 1e-12 * max(1.0, abs(ref[q]))
        full = np.zeros(n_nodes)
        for k in range(6):
            if 0 <= base + k < n_nodes:
                full[base + k] = d[k]
            else:
                assert d[k] == 0.0
        assert np.allclose(full, J[q], rtol=0, atol=1e-7)
