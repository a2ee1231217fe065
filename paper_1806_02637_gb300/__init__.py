"""GB300 epipolar-consistency (ECC) library: Python binding of libecc.so.

Thin argument marshalling over the C ABI declared in include/ecc.h; every step of
the computation runs in the library's CUDA kernels.  PyTorch is used only for
device memory and streams.  There is no CPU fallback: if the library is missing
or no GPU is present the calls raise.

Entry points (same names as the C ABI):
    ecc_precompute_radon_derivative  S_lambda of every projection (Eq. 1)
    ecc_evaluate                     d, e per pair and the total (Eq. 15-17)
    ecc_scan_consistency_host        end to end from host buffers
    ecc_status                       device-side status bits
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["EccError", "Context", "library_path", "load", "ecc_precompute_radon_derivative", "ecc_evaluate",
           "ecc_evaluate_grad", "ecc_evaluate_grad_projection", "ecc_evaluate_frozen", "ecc_evaluate_noalloc", "consistency",
           "ecc_scan_consistency_host", "ecc_status", "ecc_kernel_launches", "ecc_profile_enable",
           "ecc_profile_read", "ecc_job_footprint", "ecc_submit", "ecc_poll", "ecc_serve_stats", "ecc_serve_times",
           "ECC_F32", "ECC_F16", "ECC_BF16"]

ECC_F32, ECC_F16, ECC_BF16 = 0, 1, 2
ECC_OK = 0

_lock = threading.Lock()
_lib = None
ECC_EPENDING = 1


class _Job(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int), ("P", ctypes.c_void_p), ("motion0", ctypes.c_void_p),
                ("images", ctypes.c_void_p), ("W", ctypes.c_int), ("H", ctypes.c_int), ("n_alpha", ctypes.c_int),
                ("n_s", ctypes.c_int), ("dtype", ctypes.c_int), ("n_kappa", ctypes.c_int),
                ("cauchy_c", ctypes.c_double), ("n_iters", ctypes.c_int), ("step", ctypes.c_double),
                ("motion_out", ctypes.c_void_p), ("totals_out", ctypes.c_void_p), ("motion_model", ctypes.c_int),
                ("n_nodes", ctypes.c_int), ("param_mask", ctypes.c_int), ("nodes_out", ctypes.c_void_p),
                ("nodes0", ctypes.c_void_p)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("total_first", ctypes.c_double),
                ("total_last", ctypes.c_double), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("footprint_bytes", ctypes.c_size_t), ("line_pairs", ctypes.c_longlong), ("flags", ctypes.c_int)]


class EccError(RuntimeError):
    pass


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Loads libecc.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.SO):
            raise EccError(f"libecc.so is not built ({_build.SO})")
        lib = ctypes.CDLL(_build.SO)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        lib.ecc_version.restype = i
        lib.ecc_create.argtypes = [ctypes.POINTER(vp), i, sz]
        lib.ecc_create.restype = i
        lib.ecc_destroy.argtypes = [vp]
        lib.ecc_destroy.restype = None
        lib.ecc_last_error.argtypes = [vp]
        lib.ecc_last_error.restype = ctypes.c_char_p
        lib.ecc_status.argtypes = [vp, vp, ctypes.POINTER(i)]
        lib.ecc_status.restype = i
        lib.ecc_precompute_radon_derivative.argtypes = [vp, i, vp, vp, i, i, i, i, i, vp, vp, vp]
        lib.ecc_precompute_radon_derivative.restype = i
        lib.ecc_evaluate.argtypes = [vp, i, vp, vp, vp, vp, i, i, i, i, i, i, d, vp, i, vp, vp, vp, vp]
        lib.ecc_evaluate.restype = i
        lib.ecc_scan_consistency_host.argtypes = [vp, i, vp, vp, i, i, i, i, i, d, ctypes.POINTER(d), vp]
        lib.ecc_scan_consistency_host.restype = i
        lib.ecc_evaluate_grad.argtypes = [vp, i, vp, vp, vp, vp, i, i, i, i, i, i, d, vp, i, vp, vp, vp, vp, vp]
        lib.ecc_evaluate_grad.restype = i
        lib.ecc_evaluate_grad_projection.argtypes = [vp, i, vp, vp, vp, vp, i, i, i, i, i, i, d, vp, i, vp, vp, vp,
                                                     vp, vp]
        lib.ecc_evaluate_grad_projection.restype = i
        lib.ecc_evaluate_noalloc.argtypes = [i, vp, vp, vp, vp, i, i, i, i, i, i, d, vp, i, vp, vp, vp, vp,
                                             ctypes.c_char_p, sz]
        lib.ecc_evaluate_noalloc.restype = i
        lib.ecc_evaluate_frozen.argtypes = [vp, i, vp, vp, vp, vp, i, i, i, i, i, i, d, vp, i, vp, vp, vp, vp]
        lib.ecc_evaluate_frozen.restype = i
        lib.ecc_kernel_launches.argtypes = [vp]
        lib.ecc_kernel_launches.restype = ctypes.c_longlong
        lib.ecc_profile_enable.argtypes = [vp, i]
        lib.ecc_profile_enable.restype = i
        lib.ecc_profile_read.argtypes = [vp, vp, i, ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(d), ctypes.POINTER(i)]
        lib.ecc_profile_read.restype = i
        lib.ecc_job_footprint.argtypes = [ctypes.POINTER(_Job), ctypes.POINTER(sz)]
        lib.ecc_job_footprint.restype = i
        lib.ecc_submit.argtypes = [vp, ctypes.POINTER(_Job), ctypes.POINTER(ctypes.c_uint64)]
        lib.ecc_submit.restype = i
        lib.ecc_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(_Result)]
        lib.ecc_poll.restype = i
        lib.ecc_serve_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]
        lib.ecc_serve_stats.restype = i
        lib.ecc_serve_times.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]
        lib.ecc_serve_times.restype = i
        _lib = lib
        return lib


def _torch():
    import torch
    return torch


def _dtype_code(dt) -> int:
    torch = _torch()
    table = {torch.float32: ECC_F32, torch.float16: ECC_F16, torch.bfloat16: ECC_BF16}
    if dt not in table:
        raise EccError(f"unsupported sinogram dtype {dt}")
    return table[dt]


def _check(ctx, rc, what):
    if rc != ECC_OK:
        msg = load().ecc_last_error(ctx.handle if ctx is not None else None)
        raise EccError(f"{what} failed ({rc}): {msg.decode() if msg else ''}")


def _dev(t, dtype, name, shape=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise EccError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise EccError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise EccError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise EccError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns a library context (device scratch memory) on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        rc = lib.ecc_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
        if rc != ECC_OK:
            msg = lib.ecc_last_error(None)
            raise EccError(f"ecc_create failed ({rc}): {msg.decode() if msg else ''}")
        self.handle = h
        self.device = int(device)
        self._jobs = {}  # ticket -> host arrays of a served job (kept alive until polled)

    def close(self):
        if getattr(self, "handle", None):
            load().ecc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ecc_precompute_radon_derivative(ctx: Context, P, images, n_alpha: int, n_s: int, dtype=None, out=None,
                                    scales=None, stream=None):
    """S_lambda on the (alpha, s) grid for every view.  P: CUDA float64 [N,3,4];
    images: CUDA float32 [N,H,W].  Returns (sino [N,n_alpha,n_s], scales or None)."""
    torch = _torch()
    dtype = dtype or torch.float32
    code = _dtype_code(dtype)
    images = _dev(images, torch.float32, "images")
    N, H, W = images.shape
    P = _dev(P, torch.float64, "P", (N, 3, 4))
    if out is None:
        out = torch.empty((N, n_alpha, n_s), dtype=dtype, device=images.device)
    _dev(out, dtype, "out", (N, n_alpha, n_s))
    if code == ECC_F16:
        if scales is None:
            scales = torch.empty((N,), dtype=torch.float32, device=images.device)
        _dev(scales, torch.float32, "scales", (N,))
    else:
        scales = None
    rc = load().ecc_precompute_radon_derivative(ctx.handle, N, _ptr(P), _ptr(images), W, H, int(n_alpha), int(n_s),
                                                code, _ptr(out), _ptr(scales), _stream(stream))
    _check(ctx, rc, "ecc_precompute_radon_derivative")
    return out, scales


def _eval_args(P, sino, motion, pairs, scales, total, per_pair, nkappa, want_per_pair):
    torch = _torch()
    code = _dtype_code(sino.dtype)
    N = sino.shape[0]
    sino = _dev(sino, sino.dtype, "sino")
    P = _dev(P, torch.float64, "P", (N, 3, 4))
    dev = sino.device
    if motion is not None:
        motion = _dev(motion, torch.float64, "motion", (N, 6))
    if pairs is not None:
        pairs = _dev(pairs, torch.int32, "pairs")
        if pairs.dim() != 2 or pairs.shape[1] != 2:
            raise EccError("pairs must be [n_pairs, 2]")
        n_pairs = pairs.shape[0]
    else:
        n_pairs = N * (N - 1) // 2
    scales = _dev(scales, torch.float32, "scales", (N,)) if code == ECC_F16 else None
    if total is None:
        total = torch.empty((1,), dtype=torch.float64, device=dev)
    _dev(total, torch.float64, "total", (1,))
    if want_per_pair:
        if per_pair is None:
            per_pair = torch.empty((n_pairs, 2), dtype=torch.float64, device=dev)
        if nkappa is None:
            nkappa = torch.empty((n_pairs,), dtype=torch.int32, device=dev)
        _dev(per_pair, torch.float64, "per_pair", (n_pairs, 2))
        _dev(nkappa, torch.int32, "nkappa", (n_pairs,))
    return code, N, P, sino, motion, pairs, n_pairs, scales, total, per_pair, nkappa


def ecc_evaluate(ctx: Context, P, sino, W: int, H: int, n_kappa: int, cauchy_c: float = 0.0, motion=None,
                 pairs=None, scales=None, total=None, per_pair=None, nkappa=None, want_per_pair: bool = True,
                 stream=None) -> dict:
    """Consistency over pairs (all a < b if pairs is None).  Returns CUDA tensors
    total [1] float64, per_pair [n_pairs, 2] float64 (d, e) and nkappa [n_pairs] int32."""
    code, N, P, sino, motion, pairs, n_pairs, scales, total, per_pair, nkappa = _eval_args(
        P, sino, motion, pairs, scales, total, per_pair, nkappa, want_per_pair)
    rc = load().ecc_evaluate(ctx.handle, N, _ptr(P), _ptr(motion), _ptr(sino), _ptr(scales), int(W), int(H),
                             sino.shape[1], sino.shape[2], code, int(n_kappa), float(cauchy_c), _ptr(pairs),
                             int(n_pairs), _ptr(total), _ptr(per_pair), _ptr(nkappa), _stream(stream))
    _check(ctx, rc, "ecc_evaluate")
    return {"total": total, "per_pair": per_pair, "nkappa": nkappa}


def ecc_evaluate_frozen(ctx: Context, P, sino, W: int, H: int, n_kappa: int, cauchy_c: float = 0.0, motion=None,
                        pairs=None, scales=None, total=None, per_pair=None, nkappa=None,
                        want_per_pair: bool = True, stream=None) -> dict:
    """As ecc_evaluate with the planes sampled by the previous call on ctx (for
    finite-difference checks of the gradient); pass the same pairs tensor."""
    code, N, P, sino, motion, pairs, n_pairs, scales, total, per_pair, nkappa = _eval_args(
        P, sino, motion, pairs, scales, total, per_pair, nkappa, want_per_pair)
    rc = load().ecc_evaluate_frozen(ctx.handle, N, _ptr(P), _ptr(motion), _ptr(sino), _ptr(scales), int(W), int(H),
                                    sino.shape[1], sino.shape[2], code, int(n_kappa), float(cauchy_c), _ptr(pairs),
                                    int(n_pairs), _ptr(total), _ptr(per_pair), _ptr(nkappa), _stream(stream))
    _check(ctx, rc, "ecc_evaluate_frozen")
    return {"total": total, "per_pair": per_pair, "nkappa": nkappa}


def ecc_evaluate_noalloc(P, sino, W: int, H: int, n_kappa: int, total, cauchy_c: float = 0.0, motion=None,
                         pairs=None, scales=None, per_pair=None, nkappa=None, stream=None) -> dict:
    """ecc_evaluate without a context and without device allocation: the caller
    passes every output (total [1] float64; per_pair [n_pairs, 2] float64 and
    nkappa [n_pairs] int32 optional) and the library uses its static scratch.
    Runs on the device of sino.  Calls on one device must not overlap on the GPU."""
    torch = _torch()
    code = _dtype_code(sino.dtype)
    N = sino.shape[0]
    _dev(sino, sino.dtype, "sino")
    _dev(P, torch.float64, "P", (N, 3, 4))
    if motion is not None:
        _dev(motion, torch.float64, "motion", (N, 6))
    if pairs is not None:
        _dev(pairs, torch.int32, "pairs")
        if pairs.dim() != 2 or pairs.shape[1] != 2:
            raise EccError("pairs must be [n_pairs, 2]")
        n_pairs = pairs.shape[0]
    else:
        n_pairs = N * (N - 1) // 2
    if code == ECC_F16:
        _dev(scales, torch.float32, "scales", (N,))
    else:
        scales = None
    _dev(total, torch.float64, "total", (1,))
    if per_pair is not None:
        _dev(per_pair, torch.float64, "per_pair", (n_pairs, 2))
    if nkappa is not None:
        _dev(nkappa, torch.int32, "nkappa", (n_pairs,))
    for name, t in (("P", P), ("motion", motion), ("pairs", pairs), ("scales", scales), ("total", total),
                    ("per_pair", per_pair), ("nkappa", nkappa)):
        if t is not None and t.device != sino.device:
            raise EccError(f"{name} is on {t.device}, sino on {sino.device}: all tensors must be on one device")
    err = ctypes.create_string_buffer(512)
    with torch.cuda.device(sino.device):
        rc = load().ecc_evaluate_noalloc(N, _ptr(P), _ptr(motion), _ptr(sino), _ptr(scales), int(W), int(H),
                                         sino.shape[1], sino.shape[2], code, int(n_kappa), float(cauchy_c),
                                         _ptr(pairs), int(n_pairs), _ptr(total), _ptr(per_pair), _ptr(nkappa),
                                         _stream(stream), err, len(err))
    if rc != ECC_OK:
        raise EccError(f"ecc_evaluate_noalloc failed ({rc}): {err.value.decode()}")
    return {"total": total, "per_pair": per_pair, "nkappa": nkappa}


def ecc_evaluate_grad(ctx: Context, P, sino, W: int, H: int, n_kappa: int, cauchy_c: float = 0.0, motion=None,
                      pairs=None, scales=None, total=None, per_pair=None, nkappa=None, grad=None,
                      want_per_pair: bool = True, stream=None) -> dict:
    """As ecc_evaluate plus grad [N, 6] float64 = d total / d motion (sampled planes
    held at the evaluation point)."""
    torch = _torch()
    code, N, P, sino, motion, pairs, n_pairs, scales, total, per_pair, nkappa = _eval_args(
        P, sino, motion, pairs, scales, total, per_pair, nkappa, want_per_pair)
    if grad is None:
        grad = torch.empty((N, 6), dtype=torch.float64, device=sino.device)
    _dev(grad, torch.float64, "grad", (N, 6))
    rc = load().ecc_evaluate_grad(ctx.handle, N, _ptr(P), _ptr(motion), _ptr(sino), _ptr(scales), int(W), int(H),
                                  sino.shape[1], sino.shape[2], code, int(n_kappa), float(cauchy_c), _ptr(pairs),
                                  int(n_pairs), _ptr(total), _ptr(per_pair), _ptr(nkappa), _ptr(grad),
                                  _stream(stream))
    _check(ctx, rc, "ecc_evaluate_grad")
    return {"total": total, "per_pair": per_pair, "nkappa": nkappa, "grad": grad}


def ecc_evaluate_grad_projection(ctx: Context, P, sino, W: int, H: int, n_kappa: int, cauchy_c: float = 0.0,
                                 motion=None, pairs=None, scales=None, total=None, per_pair=None, nkappa=None,
                                 grad_P=None, want_per_pair: bool = True, stream=None) -> dict:
    """As ecc_evaluate plus grad_P [N, 12] float64 = d total / d P (entries of each
    view's projection matrix, row-major; sampled planes held at the evaluation
    point): geometric calibration by the consistency."""
    torch = _torch()
    code, N, P, sino, motion, pairs, n_pairs, scales, total, per_pair, nkappa = _eval_args(
        P, sino, motion, pairs, scales, total, per_pair, nkappa, want_per_pair)
    if grad_P is None:
        grad_P = torch.empty((N, 12), dtype=torch.float64, device=sino.device)
    _dev(grad_P, torch.float64, "grad_P", (N, 12))
    rc = load().ecc_evaluate_grad_projection(ctx.handle, N, _ptr(P), _ptr(motion), _ptr(sino), _ptr(scales),
                                             int(W), int(H), sino.shape[1], sino.shape[2], code, int(n_kappa),
                                             float(cauchy_c), _ptr(pairs), int(n_pairs), _ptr(total),
                                             _ptr(per_pair), _ptr(nkappa), _ptr(grad_P), _stream(stream))
    _check(ctx, rc, "ecc_evaluate_grad_projection")
    return {"total": total, "per_pair": per_pair, "nkappa": nkappa, "grad_P": grad_P}


def _autograd_function():
    torch = _torch()

    class _Consistency(torch.autograd.Function):
        """total(motion) with the adjoint kernel as backward."""

        @staticmethod
        def forward(fctx, motion, ctx, P, sino, W, H, n_kappa, cauchy_c, pairs, scales):
            motion = motion.detach().contiguous()
            if motion.requires_grad or fctx.needs_input_grad[0]:
                r = ecc_evaluate_grad(ctx, P, sino, W, H, n_kappa, cauchy_c, motion=motion, pairs=pairs,
                                      scales=scales, want_per_pair=False)
                fctx.save_for_backward(r["grad"])
            else:
                r = ecc_evaluate(ctx, P, sino, W, H, n_kappa, cauchy_c, motion=motion, pairs=pairs, scales=scales,
                                 want_per_pair=False)
                fctx.save_for_backward(torch.zeros_like(motion))
            return r["total"][0].clone()

        @staticmethod
        def backward(fctx, g):
            (grad,) = fctx.saved_tensors
            return (g * grad, None, None, None, None, None, None, None, None, None)

    return _Consistency


_FN = None


def consistency(ctx: Context, motion, P, sino, W: int, H: int, n_kappa: int, cauchy_c: float = 0.0, pairs=None,
                scales=None):
    """Differentiable total (Eq. 17) as a function of the per-view motion [N, 6]
    (torch.autograd.Function; backward = the library's adjoint kernel)."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(motion, ctx, P, sino, W, H, n_kappa, cauchy_c, pairs, scales)


def ecc_scan_consistency_host(ctx: Context, P, images, n_alpha: int, n_s: int, n_kappa: int,
                              cauchy_c: float = 0.0, stream=None) -> float:
    """End to end from host arrays (numpy or CPU tensors; pinned tensors copy faster)."""
    torch = _torch()
    if isinstance(P, torch.Tensor):
        P = P.detach().cpu().numpy()
    P = np.ascontiguousarray(P, dtype=np.float64)
    if isinstance(images, torch.Tensor):
        if images.is_cuda or images.dtype != torch.float32 or not images.is_contiguous():
            raise EccError("images must be a contiguous CPU float32 tensor")
        img_ptr, shape = images.data_ptr(), tuple(images.shape)
    else:
        images = np.ascontiguousarray(images, dtype=np.float32)
        img_ptr, shape = images.ctypes.data, images.shape
    N, H, W = shape
    if P.shape != (N, 3, 4):
        raise EccError("P must be [N, 3, 4]")
    out = ctypes.c_double(0.0)
    rc = load().ecc_scan_consistency_host(ctx.handle, N, ctypes.c_void_p(P.ctypes.data), ctypes.c_void_p(img_ptr),
                                          W, H, int(n_alpha), int(n_s), int(n_kappa), float(cauchy_c),
                                          ctypes.byref(out), _stream(stream))
    _check(ctx, rc, "ecc_scan_consistency_host")
    return out.value


def ecc_status(ctx: Context, stream=None) -> int:
    flags = ctypes.c_int(0)
    rc = load().ecc_status(ctx.handle, _stream(stream), ctypes.byref(flags))
    _check(ctx, rc, "ecc_status")
    return flags.value


def ecc_kernel_launches(ctx: Context) -> int:
    """Number of kernels the context has launched so far."""
    return int(load().ecc_kernel_launches(ctx.handle))


def ecc_profile_enable(ctx: Context, enable: bool = True) -> None:
    _check(ctx, load().ecc_profile_enable(ctx.handle, int(bool(enable))), "ecc_profile_enable")


def ecc_profile_read(ctx: Context, stream=None, max_entries: int = 32) -> dict:
    """{kernel name: (launches, summed ms)} since the last read (waits for the stream)."""
    names = ctypes.create_string_buffer(32 * max_entries)
    launches = (ctypes.c_longlong * max_entries)()
    ms = (ctypes.c_double * max_entries)()
    n = ctypes.c_int(0)
    rc = load().ecc_profile_read(ctx.handle, _stream(stream), max_entries, names, launches, ms, ctypes.byref(n))
    _check(ctx, rc, "ecc_profile_read")
    out = {}
    for k in range(n.value):
        nm = names.raw[32 * k:32 * (k + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[k]), float(ms[k]))
    return out


# ---------------------------------------------------------------- serving
_DT = {"float32": ECC_F32, "float16": ECC_F16, "bfloat16": ECC_BF16}
_MODELS = {"per_view": 0, "akima": 1}


def _host_array(a, dtype, name, shape):
    """Host array for a job: numpy or CPU torch tensor (pinned memory is used as is)."""
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise EccError(f"{name} must be in host memory")
        if a.dtype != getattr(torch, np.dtype(dtype).name) or not a.is_contiguous():
            raise EccError(f"{name} must be a contiguous {np.dtype(dtype).name} tensor")
        ptr = a.data_ptr()
    else:
        a = np.ascontiguousarray(a, dtype=dtype)
        ptr = a.ctypes.data
    if tuple(a.shape) != tuple(shape):
        raise EccError(f"{name} has shape {tuple(a.shape)}, expected {tuple(shape)}")
    return a, ptr


def _job_struct(P, images, W, H, n_alpha, n_s, n_kappa, n_iters, step, dtype, cauchy_c, motion0,
                motion_model="per_view", n_nodes=0, param_mask=0, nodes0=None):
    n = int(P.shape[0])
    P, p_ptr = _host_array(P, np.float64, "P", (n, 3, 4))
    images, i_ptr = _host_array(images, np.float32, "images", (n, H, W))
    m_ptr = None
    if motion0 is not None:
        motion0, m_ptr = _host_array(motion0, np.float64, "motion0", (n, 6))
    code = _DT[dtype] if isinstance(dtype, str) else _dtype_code(dtype)
    motion_out = np.zeros((n, 6))
    totals_out = np.zeros(int(n_iters) + 1)
    model = _MODELS[motion_model] if isinstance(motion_model, str) else int(motion_model)
    nodes_out = np.zeros((max(int(n_nodes), 1), 6))
    n0_ptr = None
    if nodes0 is not None:
        nodes0, n0_ptr = _host_array(nodes0, np.float64, "nodes0", (int(n_nodes), 6))
    j = _Job(n, p_ptr, m_ptr, i_ptr, int(W), int(H), int(n_alpha), int(n_s), code, int(n_kappa), float(cauchy_c),
             int(n_iters), float(step), motion_out.ctypes.data, totals_out.ctypes.data, model, int(n_nodes),
             int(param_mask), nodes_out.ctypes.data, n0_ptr)
    return j, (P, images, motion0, motion_out, totals_out, nodes_out, nodes0)


def ecc_job_footprint(P, images, W: int, H: int, n_alpha: int, n_s: int, n_kappa: int, n_iters: int = 20,
                      step: float = 0.0, dtype="float32", cauchy_c: float = 0.0, motion0=None,
                      motion_model="per_view", n_nodes: int = 0, param_mask: int = 0) -> int:
    """Device bytes the job holds while admitted."""
    j, _ = _job_struct(P, images, W, H, n_alpha, n_s, n_kappa, n_iters, step, dtype, cauchy_c, motion0,
                       motion_model, n_nodes, param_mask)
    b = ctypes.c_size_t(0)
    rc = load().ecc_job_footprint(ctypes.byref(j), ctypes.byref(b))
    _check(None, rc, "ecc_job_footprint")
    return int(b.value)


def ecc_submit(ctx: Context, P, images, W: int, H: int, n_alpha: int, n_s: int, n_kappa: int, n_iters: int = 20,
               step: float = 0.0, dtype="float32", cauchy_c: float = 0.0, motion0=None, motion_model="per_view",
               n_nodes: int = 0, param_mask: int = 0, nodes0=None) -> int:
    """Queues a motion-compensation job (host P [n,3,4] float64, images [n,H,W] float32,
    optional motion0 [n,6]); returns its ticket.  motion_model "per_view" estimates the
    parameters of every view, "akima" the n_nodes node values of an Akima spline per
    parameter over the view index (added to motion0; initial node values nodes0
    [n_nodes, 6] or zeros); param_mask selects the estimated parameters (bits of rx,
    ry, rz, tx, ty, tz; 0 = all).  The host arrays are kept alive by the context until
    the job is polled."""
    j, keep = _job_struct(P, images, W, H, n_alpha, n_s, n_kappa, n_iters, step, dtype, cauchy_c, motion0,
                          motion_model, n_nodes, param_mask, nodes0)
    t = ctypes.c_uint64(0)
    rc = load().ecc_submit(ctx.handle, ctypes.byref(j), ctypes.byref(t))
    _check(ctx, rc, "ecc_submit")
    ctx._jobs[int(t.value)] = keep
    return int(t.value)


def ecc_poll(ctx: Context, ticket: int):
    """None while the job is pending; otherwise a dict with the result record, the
    final motion [n,6] and the totals [n_iters + 1] (raises EccError if the job failed)."""
    r = _Result()
    rc = load().ecc_poll(ctx.handle, ctypes.c_uint64(ticket), ctypes.byref(r))
    if rc == ECC_EPENDING:
        return None
    keep = ctx._jobs.pop(int(ticket), None)
    _check(ctx, rc, "ecc_poll")
    out = {k: getattr(r, k) for k, _ in _Result._fields_}
    if keep is not None:
        out["motion"] = keep[3]
        out["totals"] = keep[4]
        out["nodes"] = keep[5]
    return out


def ecc_serve_stats(ctx: Context) -> dict:
    rounds, job_rounds, lp = ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_longlong(0)
    mb = ctypes.c_int(0)
    rc = load().ecc_serve_stats(ctx.handle, ctypes.byref(rounds), ctypes.byref(job_rounds), ctypes.byref(mb),
                                ctypes.byref(lp))
    _check(ctx, rc, "ecc_serve_stats")
    return {"rounds": rounds.value, "job_rounds": job_rounds.value, "max_batch": mb.value, "line_pairs": lp.value}


def ecc_serve_times(ctx: Context) -> dict:
    """Serving device time [ms]: input uploads, precomputes and rounds (CUDA events)."""
    up, pre, rnd = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    rc = load().ecc_serve_times(ctx.handle, ctypes.byref(up), ctypes.byref(pre), ctypes.byref(rnd))
    _check(ctx, rc, "ecc_serve_times")
    return {"upload_ms": up.value, "precompute_ms": pre.value, "round_ms": rnd.value}
