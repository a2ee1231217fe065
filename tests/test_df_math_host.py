"""The double-float sin/cos and atan2 of the per-pair set-up (csrc/df.cuh), run on the
CPU through an internal host entry point, against FP64 library values: errors near
the double-float unit (2^-44 relative to the operands), over the argument ranges the
set-up uses (sin/cos of |x| <= 4, atan2 of any direction, including the axes and
arguments of very different magnitude)."""
import ctypes

import numpy as np

from paper_1806_02637_gb300 import build as ecc_build

_dp = ctypes.POINTER(ctypes.c_double)


def _f():
    lib = ctypes.CDLL(ecc_build.build())
    f = lib.ecc_internal_df_math_host
    f.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _dp]
    f.restype = ctypes.c_int
    return f


def _sincos(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2 * len(x))
    assert _f()(0, x.ctypes.data_as(_dp), None, len(x), out.ctypes.data_as(_dp)) == 0
    return out[0::2], out[1::2]


def _atan2(y, x):
    y, x = (np.ascontiguousarray(a, dtype=np.float64) for a in (y, x))
    out = np.zeros(len(y))
    assert _f()(1, y.ctypes.data_as(_dp), x.ctypes.data_as(_dp), len(y), out.ctypes.data_as(_dp)) == 0
    return out


def test_df_sincos_against_fp64():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-4.0, 4.0, 20000), rng.uniform(-1e-3, 1e-3, 2000),
                        np.array([0.0, np.pi / 4, np.pi / 2, np.pi, -np.pi, 3.0, -3.9, 1e-12])])
    s, c = _sincos(x)
    assert np.abs(s - np.sin(x)).max() < 2e-14
    assert np.abs(c - np.cos(x)).max() < 2e-14
    small = np.abs(x) < 1e-3  # relative accuracy where the value is small
    assert (np.abs(s - np.sin(x))[small] <= 1e-13 * np.abs(x[small]) + 1e-30).all()


def test_df_atan2_against_fp64():
    rng = np.random.default_rng(4)
    ang = rng.uniform(-np.pi, np.pi, 20000)
    r = np.exp(rng.uniform(-20.0, 20.0, ang.size))
    y, x = r * np.sin(ang), r * np.cos(ang)
    extra_y = np.array([1.0, -1.0, 0.0, 1e-9, 5.0, -3e6, 1e-20])
    extra_x = np.array([0.0, 0.0, 1.0, -1.0, 5.0, 1e-3, 1.0])
    y, x = np.concatenate([y, extra_y]), np.concatenate([x, extra_x])
    got, want = _atan2(y, x), np.arctan2(y, x)
    d = np.abs(got - want)
    d = np.minimum(d, 2 * np.pi - d)  # the branch cut at +-pi
    assert d.max() < 3e-14, d.max()
    assert _atan2(np.zeros(1), np.zeros(1))[0] == 0.0
