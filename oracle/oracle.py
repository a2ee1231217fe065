"""ctypes wrapper of the FP64 CPU oracle (``ecc_oracle.c``).

TEST INFRASTRUCTURE ONLY: used by the tests, by the smoke check and by the
benchmark's CPU-baseline leg.  The product path never imports this module and
the CUDA library shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SOURCES = ["ecc_oracle.c", "ecc_pair_generic.h"]
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile the oracle (plain C99, FP64, no fast-math, no FMA contraction)."""
    newest = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SOURCES)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-pthread", "-o", tmp, os.path.join(_HERE, "ecc_oracle.c"), "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_meet.argtypes = [_dp, _dp, _dp]
            lib.orc_dual.argtypes = [_dp, ctypes.c_int, _dp]
            lib.orc_source.argtypes = [_dp, _dp]
            lib.orc_line_inf.argtypes = [_dp, _dp, _dp]
            lib.orc_line_pinv.argtypes = [_dp, _dp, _dp]
            lib.orc_line_pinv.restype = ctypes.c_int
            lib.orc_apply_motion.argtypes = [_dp, _dp, _dp]
            lib.orc_view_setup.argtypes = [_dp, _dp, _dp]
            lib.orc_view_setup.restype = ctypes.c_int
            lib.orc_pair_arcs.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp]
            lib.orc_pair_arcs.restype = ctypes.c_int
            lib.orc_pair_frame.argtypes = [_dp, _dp, _dp, _dp]
            lib.orc_pair_frame.restype = ctypes.c_int
            lib.orc_lookup.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _ip]
            lib.orc_lookup.restype = ctypes.c_double
            lib.orc_radon_derivative.argtypes = [ctypes.c_int, _dp, _fp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, _dp]
            lib.orc_radon_derivative.restype = ctypes.c_int
            ecc_args = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                        ctypes.c_int, ctypes.c_double, _ip, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                        _dp, _dp, _ip, _dp]
            lib.orc_ecc.argtypes = ecc_args + [_ip, _dp]
            lib.orc_ecc.restype = ctypes.c_int
            lib.orc_ecc_grad.argtypes = ecc_args + [_dp, _dp]
            lib.orc_ecc_grad.restype = ctypes.c_int
            lib.orc_ecc_grad_P.argtypes = ecc_args + [_dp, _dp]
            lib.orc_ecc_grad_P.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, kind=_dp):
    return None if a is None else a.ctypes.data_as(kind)


def _threads(n_threads):
    return int(n_threads or os.cpu_count() or 1)


def meet(a, b) -> np.ndarray:
    """Eq. (4): Pluecker coordinates (p, q, r, s, t, u) of the meet of planes a, b."""
    a, b, L = _d(a), _d(b), np.zeros(6)
    _load().orc_meet(_ptr(a), _ptr(b), _ptr(L))
    return L


def dual(L, corrected: bool = True) -> np.ndarray:
    """Eq. (5): dual line matrix L_K (4x4); corrected selects the sign reading."""
    L, K = _d(L), np.zeros(16)
    _load().orc_dual(_ptr(L), int(bool(corrected)), _ptr(K))
    return K.reshape(4, 4)


def source(P) -> np.ndarray:
    """Homogeneous source position: meet of the three rows of P."""
    P, X = _d(P).reshape(12), np.zeros(4)
    _load().orc_source(_ptr(P), _ptr(X))
    return X


def line_inf(P, E) -> np.ndarray:
    """Eq. (13)/(14): epipolar line of plane E through its line at infinity."""
    P, E, l = _d(P).reshape(12), _d(E), np.zeros(3)
    _load().orc_line_inf(_ptr(P), _ptr(E), _ptr(l))
    return l


def line_pinv(P, E) -> np.ndarray:
    """Prior method: l = P^{+T} E (P normalised to det M > 0 by the caller)."""
    P, E, l = _d(P).reshape(12), _d(E), np.zeros(3)
    if _load().orc_line_pinv(_ptr(P), _ptr(E), _ptr(l)) != 0:
        raise ValueError("singular P P^T")
    return l


def apply_motion(P, theta) -> np.ndarray:
    """P T(theta), theta = (rx, ry, rz, tx, ty, tz)."""
    P, th, out = _d(P).reshape(12), _d(theta), np.zeros(12)
    _load().orc_apply_motion(_ptr(P), _ptr(th), _ptr(out))
    return out.reshape(3, 4)


def view_setup(P, theta=None) -> dict:
    """Normalised P, source C and up axis of one view."""
    P, out = _d(P).reshape(12), np.zeros(18)
    th = None if theta is None else _d(theta)
    if _load().orc_view_setup(_ptr(P), _ptr(th), _ptr(out)) != 0:
        raise ValueError("degenerate projection matrix")
    return {"P": out[:12].reshape(3, 4), "C": out[12:15], "up": out[15:18]}


def pair_frame(Pa, Pb):
    w, v = np.zeros(3), np.zeros(3)
    Pa, Pb = _d(Pa).reshape(12), _d(Pb).reshape(12)
    if _load().orc_pair_frame(_ptr(Pa), _ptr(Pb), _ptr(w), _ptr(v)) != 0:
        raise ValueError("coincident sources")
    return w, v


def pair_arcs(Pa, Pb, W, H, tha=None, thb=None) -> np.ndarray:
    """{sampled view, lo_s, len_s, lo_o, len_o} of one pair."""
    out = np.zeros(5)
    Pa, Pb = _d(Pa).reshape(12), _d(Pb).reshape(12)
    tha = None if tha is None else _d(tha)
    thb = None if thb is None else _d(thb)
    if _load().orc_pair_arcs(_ptr(Pa), _ptr(Pb), _ptr(tha), _ptr(thb), int(W), int(H), _ptr(out)) != 0:
        raise ValueError("degenerate pair")
    return out


def lookup(sino, W, H, l):
    """S at detector line l of one view's sinogram [n_alpha, n_s]; returns (value, hit)."""
    sino = _d(sino)
    l = _d(l)
    hit = ctypes.c_int(0)
    v = _load().orc_lookup(_ptr(sino), sino.shape[0], sino.shape[1], int(W), int(H), _ptr(l), ctypes.byref(hit))
    return v, bool(hit.value)


def radon_derivative(P, images, n_alpha: int, n_s: int, n_threads=None) -> np.ndarray:
    """S_lambda on the (alpha, s) grid for every view: [n_views, n_alpha, n_s] FP64."""
    P = _d(P).reshape(-1, 12)
    images = np.ascontiguousarray(images, dtype=np.float32)
    nv, H, W = images.shape
    assert P.shape[0] == nv
    out = np.zeros((nv, n_alpha, n_s))
    rc = _load().orc_radon_derivative(nv, _ptr(P), _ptr(images, _fp), W, H, int(n_alpha), int(n_s),
                                      _threads(n_threads), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_radon_derivative failed ({rc})")
    return out


def _pairs_arg(pairs, n_views):
    if pairs is None:
        a, b = np.triu_indices(n_views, k=1)
        pairs = np.stack([a, b], axis=1)
    return np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)


def ecc(P, sino, W: int, H: int, K: int, cauchy_c: float = 0.0, motion=None, pairs=None,
        construction: str = "inf", arcs=None, n_threads=None) -> dict:
    """Eq. (15)-(17) over the pairs.  sino [n_views, n_alpha, n_s] (values used in FP64).

    Returns d, e, nk per pair, the arcs used, the count of samples whose two validity
    tests disagree, and the total.  ``arcs`` freezes the sampled arcs (validity then
    by arc membership)."""
    P = _d(P).reshape(-1, 12)
    nv = P.shape[0]
    sino = _d(sino)
    assert sino.shape[0] == nv
    pr = _pairs_arg(pairs, nv)
    npairs = pr.shape[0]
    mot = None if motion is None else _d(motion).reshape(nv, 6)
    arcs_in = None if arcs is None else _d(arcs).reshape(npairs, 5)
    d, e = np.zeros(npairs), np.zeros(npairs)
    nk = np.zeros(npairs, dtype=np.int32)
    mm = np.zeros(npairs, dtype=np.int32)
    arcs_out = np.zeros((npairs, 5))
    total = ctypes.c_double(0.0)
    cons = {"inf": 0, "pinv": 1}[construction]
    rc = _load().orc_ecc(nv, _ptr(P), _ptr(mot), _ptr(sino), int(W), int(H), sino.shape[1], sino.shape[2], int(K),
                         float(cauchy_c), _ptr(pr, _ip), npairs, cons, _ptr(arcs_in), _threads(n_threads),
                         _ptr(d), _ptr(e), _ptr(nk, _ip), _ptr(arcs_out), _ptr(mm, _ip), ctypes.byref(total))
    if rc != 0:
        raise RuntimeError(f"orc_ecc failed ({rc})")
    return {"d": d, "e": e, "nk": nk, "arcs": arcs_out, "mismatch": mm, "total": total.value, "pairs": pr}


def _grad(fn, npv, P, sino, W, H, K, cauchy_c, motion, pairs, construction, arcs, n_threads):
    P = _d(P).reshape(-1, 12)
    nv = P.shape[0]
    sino = _d(sino)
    pr = _pairs_arg(pairs, nv)
    npairs = pr.shape[0]
    mot = None if motion is None else _d(motion).reshape(nv, 6)
    arcs_in = None if arcs is None else _d(arcs).reshape(npairs, 5)
    d, e = np.zeros(npairs), np.zeros(npairs)
    nk = np.zeros(npairs, dtype=np.int32)
    arcs_out = np.zeros((npairs, 5))
    grad = np.zeros((nv, npv))
    total = ctypes.c_double(0.0)
    cons = {"inf": 0, "pinv": 1}[construction]
    rc = fn(nv, _ptr(P), _ptr(mot), _ptr(sino), int(W), int(H), sino.shape[1], sino.shape[2], int(K),
            float(cauchy_c), _ptr(pr, _ip), npairs, cons, _ptr(arcs_in), _threads(n_threads), _ptr(d), _ptr(e),
            _ptr(nk, _ip), _ptr(arcs_out), ctypes.byref(total), _ptr(grad))
    if rc != 0:
        raise RuntimeError(f"oracle gradient failed ({rc})")
    return {"d": d, "e": e, "nk": nk, "arcs": arcs_out, "total": total.value, "grad": grad, "pairs": pr}


def ecc_grad(P, sino, W: int, H: int, K: int, cauchy_c: float = 0.0, motion=None, pairs=None,
             construction: str = "inf", arcs=None, n_threads=None) -> dict:
    """Gradient of the total w.r.t. per-view motion [n_views, 6] by complex-step
    differentiation, arcs and validity frozen at the evaluation point."""
    return _grad(_load().orc_ecc_grad, 6, P, sino, W, H, K, cauchy_c, motion, pairs, construction, arcs, n_threads)


def ecc_grad_P(P, sino, W: int, H: int, K: int, cauchy_c: float = 0.0, motion=None, pairs=None,
               construction: str = "inf", arcs=None, n_threads=None) -> dict:
    """Gradient of the total w.r.t. the entries of each view's projection matrix
    ("grad" [n_views, 12], row-major like P; the view uses P T(theta)) by
    complex-step differentiation, arcs and validity frozen at the evaluation point:
    geometric calibration by the consistency (Introduction)."""
    return _grad(_load().orc_ecc_grad_P, 12, P, sino, W, H, K, cauchy_c, motion, pairs, construction, arcs,
                 n_threads)
