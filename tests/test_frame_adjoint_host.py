"""The reverse mode of the pencil frame (pencil_frame_adjoint_df: the frame of the
plane pencil around the baseline and its adjoint, in double-float), run on the CPU
through an internal host entry point: the frame is orthonormal with w and v normal to
the baseline, and the gradient of a linear functional gw.w + gv.v with respect to the
source positions and the up axes matches central differences of the same code, for
distant, neighbouring and fallback-axis geometries (R3: up_a + up_b along the
baseline)."""
import ctypes

import numpy as np
import pytest

from paper_1806_02637_gb300 import build as ecc_build

_dp = ctypes.POINTER(ctypes.c_double)


def _frame(Ca, Cb, upa, upb, gw, gv):
    lib = ctypes.CDLL(ecc_build.build())
    f = lib.ecc_internal_frame_adjoint_host
    f.argtypes = [_dp] * 8
    f.restype = ctypes.c_int
    args = [np.ascontiguousarray(x, dtype=np.float64) for x in (Ca, Cb, upa, upb, gw, gv)]
    wv, grad = np.zeros(6), np.zeros(9)
    assert f(*[a.ctypes.data_as(_dp) for a in args], wv.ctypes.data_as(_dp), grad.ctypes.data_as(_dp)) == 0
    return wv[:3], wv[3:], grad


def _on_circle(deg):
    t = np.deg2rad(deg)
    return 750.0 * np.array([np.cos(t), np.sin(t), 0.0])


_B = np.array([0.3, 0.1, 1.0]) / np.linalg.norm([0.3, 0.1, 1.0])

CASES = {
    "distant": (_on_circle(10.0), _on_circle(130.0), np.array([0.0, 0.01, 1.0]), np.array([0.02, 0.0, 1.0])),
    "neighbouring": (_on_circle(40.0), _on_circle(40.4), np.array([0.0, 0.0, 1.0]), np.array([0.001, 0.0, 1.0])),
    # up_a + up_b along the baseline (2 mm): the fallback axis, here unique (the smallest
    # |u_k| is u_y alone; where two |u_k| tie, as for a baseline along z, a step of the
    # central differences would switch the axis)
    "fallback": (_on_circle(25.0), _on_circle(25.0) + 2.0 * _B, _B, _B),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_frame_adjoint_against_central_differences(case):
    Ca, Cb, upa, upb = CASES[case]
    rng = np.random.default_rng(hash(case) % 2**32)
    gw, gv = rng.normal(size=3), rng.normal(size=3)
    w, v, grad = _frame(Ca, Cb, upa, upb, gw, gv)
    u = (Cb - Ca) / np.linalg.norm(Cb - Ca)
    assert abs(np.dot(w, w) - 1) < 1e-12 and abs(np.dot(v, v) - 1) < 1e-12
    assert abs(np.dot(w, u)) < 1e-12 and abs(np.dot(v, u)) < 1e-12 and abs(np.dot(w, v)) < 1e-12

    def L(Ca_, Cb_, upa_, upb_):
        w_, v_, _ = _frame(Ca_, Cb_, upa_, upb_, gw, gv)
        return gw @ w_ + gv @ v_

    # steps: inside the fallback regime (|w_t| < 1e-6) they must keep |w_t| below the
    # threshold, where the frame switches branch
    h_c, h_up, tol = (1e-8, 1e-9, 1e-4) if case == "fallback" else (1e-3, 1e-6, 1e-6)
    fd = np.zeros(12)
    for j in range(12):
        h = h_c if j < 6 else h_up
        args_p = [Ca.copy(), Cb.copy(), upa.copy(), upb.copy()]
        args_m = [Ca.copy(), Cb.copy(), upa.copy(), upb.copy()]
        args_p[j // 3][j % 3] += h
        args_m[j // 3][j % 3] -= h
        fd[j] = (L(*args_p) - L(*args_m)) / (2 * h)
    want = np.concatenate([grad[:6], grad[6:], grad[6:]])  # d/d up_a = d/d up_b = gup
    scale = np.abs(fd).max()
    assert np.abs(want - fd).max() <= tol * scale, (want, fd)
