"""Seeded synthetic inputs for the epipolar-consistency (ECC) path.

Input generation only: circular C-arm trajectories (projection matrices), seeded
phantoms (Gaussian blobs, uniform ellipsoids) placed inside the fully visible
field of view, their analytic cone-beam projections (``project.c``) and seeded
per-view rigid motion.  Nothing here computes any part of the consistency
method; both the CPU oracle and the CUDA library consume these inputs.

The paper's own data (a 200-degree short scan of a head phantom on a robotic
C-arm, Experiments section) is not available; the presets below stand in for it
with the view count and arc of that scan and the detector sizes of the
benchmark configurations.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the analytic projector (plain C, pthreads) into synth/_build."""
    src = os.path.join(_HERE, "project.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.synth_project.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
            lib.synth_project.restype = ctypes.c_int
            lib.synth_ray_value.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int]
            lib.synth_ray_value.restype = ctypes.c_double
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclasses.dataclass(frozen=True)
class ScanConfig:
    """One synthetic scan workload (trajectory, detector, phantom, sampling)."""
    name: str
    n_views: int
    arc_deg: float
    full_scan: bool
    W: int
    H: int
    pixel_mm: float
    sid: float = 750.0
    sdd: float = 1200.0
    phantom: str = "ellipsoids"          # "blobs" or "ellipsoids"
    n_prim: int = 40
    size_range: tuple = (5.0, 80.0)      # blob sigma or ellipsoid semi-axes [mm]
    value_range: tuple = (0.1, 1.0)      # blob amplitude or ellipsoid density [1/mm]
    extent_sigmas: float = 3.0           # blob support used for untruncated placement
    n_alpha: int = 768
    n_s: int = 768
    K: int = 512
    seed: int = 1806_02637
    motion_rot_deg: float = 0.0
    motion_trans_mm: float = 0.0

    @property
    def n_pairs(self) -> int:
        return self.n_views * (self.n_views - 1) // 2


# Named workloads.  C1: two views 90 degrees apart, Gaussian blobs (small case).
# C2: full 200-degree short scan, 496 views (the paper's scan geometry), ellipsoids.
# C3: 248 views with seeded rigid motion (differentiation).  C4: 1240-view full scan
# on a 976^2 detector (reduced-precision sinogram storage).
CONFIGS = {
    "c1": ScanConfig("c1", n_views=2, arc_deg=90.0, full_scan=False, W=256, H=256, pixel_mm=1.0,
                     phantom="blobs", n_prim=3, size_range=(10.0, 30.0), value_range=(0.01, 0.02),
                     n_alpha=256, n_s=363, K=256, seed=1806_02637_1),
    "c2": ScanConfig("c2", n_views=496, arc_deg=200.0, full_scan=False, W=620, H=480, pixel_mm=0.6,
                     phantom="ellipsoids", n_prim=40, size_range=(5.0, 80.0), value_range=(0.1, 1.0),
                     n_alpha=768, n_s=768, K=512, seed=1806_02637_2),
    "c3": ScanConfig("c3", n_views=248, arc_deg=200.0, full_scan=False, W=620, H=480, pixel_mm=0.6,
                     phantom="ellipsoids", n_prim=40, size_range=(5.0, 80.0), value_range=(0.1, 1.0),
                     n_alpha=768, n_s=768, K=512, seed=1806_02637_3, motion_rot_deg=1.0, motion_trans_mm=2.0),
    "c4": ScanConfig("c4", n_views=1240, arc_deg=360.0, full_scan=True, W=976, H=976, pixel_mm=0.3,
                     phantom="ellipsoids", n_prim=60, size_range=(5.0, 80.0), value_range=(0.1, 1.0),
                     n_alpha=1024, n_s=1382, K=1024, seed=1806_02637_4),
}


def view_angles(cfg: ScanConfig) -> np.ndarray:
    """Source angles [rad]: i * arc / (N - 1) for a short scan, i * 360 / N for a full scan."""
    i = np.arange(cfg.n_views, dtype=np.float64)
    if cfg.full_scan:
        return np.deg2rad(i * 360.0 / cfg.n_views)
    return np.deg2rad(i * cfg.arc_deg / max(cfg.n_views - 1, 1))


def projection_matrix(theta: float, W: int, H: int, pixel_mm: float, sid: float, sdd: float) -> np.ndarray:
    """P = K [R | -R C] for a source at C = SID (cos t, sin t, 0) looking at the origin.

    Detector axes: r1 = (-sin t, cos t, 0) (columns), r2 = (0, 0, -1) (rows),
    viewing direction r3 = -(cos t, sin t, 0); K = [[f, 0, (W-1)/2], [0, f, (H-1)/2], [0, 0, 1]]
    with f = SDD / pixel, so pixel centres sit on integer coordinates.
    """
    c, s = np.cos(theta), np.sin(theta)
    R = np.array([[-s, c, 0.0], [0.0, 0.0, -1.0], [-c, -s, 0.0]])
    C = sid * np.array([c, s, 0.0])
    f = sdd / pixel_mm
    Kmat = np.array([[f, 0.0, 0.5 * (W - 1)], [0.0, f, 0.5 * (H - 1)], [0.0, 0.0, 1.0]])
    return Kmat @ np.hstack([R, (-R @ C)[:, None]])


def trajectory(cfg: ScanConfig) -> np.ndarray:
    """Projection matrices [n_views, 3, 4] (FP64) of the circular trajectory."""
    return np.stack([projection_matrix(t, cfg.W, cfg.H, cfg.pixel_mm, cfg.sid, cfg.sdd)
                     for t in view_angles(cfg)])


def fov(cfg: ScanConfig):
    """(r_max, z_max(r)): the cylinder seen untruncated by every view of a circle."""
    half_w = 0.5 * cfg.W * cfg.pixel_mm
    half_h = 0.5 * cfg.H * cfg.pixel_mm
    r_max = cfg.sid * np.sin(np.arctan(half_w / cfg.sdd))

    def z_max(r):
        return half_h * (cfg.sid - r) / cfg.sdd

    return r_max, z_max


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def phantom(cfg: ScanConfig, rng: np.random.Generator | None = None, margin: float = 0.97,
            max_tries: int = 200000) -> np.ndarray:
    """Seeded primitives [n_prim, 17], each placed so that its support (3 sigma for
    blobs, the exact bounding extent for ellipsoids) stays inside the untruncated
    cylinder.  Sizes are drawn from size_range and re-drawn until they fit, so the
    accepted sizes follow size_range conditioned on fitting."""
    if rng is None:
        rng = np.random.Generator(np.random.PCG64(cfg.seed))
    r_max, z_max = fov(cfg)
    r_max *= margin
    out = []
    tries = 0
    while len(out) < cfg.n_prim:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("phantom placement did not converge")
        val = rng.uniform(*cfg.value_range)
        if cfg.phantom == "blobs":
            sig = rng.uniform(*cfg.size_range)
            axes = np.array([sig, sig, sig])
            R = np.eye(3)
            ext_xy = ext_z = cfg.extent_sigmas * sig
        else:
            axes = rng.uniform(*cfg.size_range, size=3)
            R = random_rotation(rng)
            Sig = R @ np.diag(axes ** 2) @ R.T
            ext_xy = np.sqrt(np.linalg.eigvalsh(Sig[:2, :2]).max())
            ext_z = np.sqrt(Sig[2, 2])
        rc = rng.uniform(0.0, 1.0) ** 0.5 * r_max
        phi = rng.uniform(0.0, 2 * np.pi)
        zc = rng.uniform(-1.0, 1.0) * z_max(r_max) * margin
        centre = np.array([rc * np.cos(phi), rc * np.sin(phi), zc])
        r_out = rc + ext_xy
        if r_out > r_max:
            continue
        if abs(zc) + ext_z > margin * z_max(r_out):
            continue
        rec = np.zeros(17)
        rec[0] = 0.0 if cfg.phantom == "blobs" else 1.0
        rec[1] = val
        rec[2:5] = centre
        rec[5:8] = axes
        rec[8:17] = R.reshape(-1)
        out.append(rec)
    return np.stack(out)


def project(P: np.ndarray, prim: np.ndarray, W: int, H: int, n_threads: int | None = None) -> np.ndarray:
    """Analytic cone-beam projections [n_views, H, W] (FP32) of the primitives."""
    lib = _load()
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1, 12)
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    out = np.zeros((P.shape[0], H, W), dtype=np.float32)
    nt = n_threads or os.cpu_count() or 1
    lib.synth_project(P.shape[0], _dptr(P), W, H, _dptr(prim), prim.shape[0], nt,
                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return out


def ray_value(P: np.ndarray, u: float, v: float, prim: np.ndarray) -> float:
    """Line integral through continuous detector coordinate (u, v) of one view."""
    lib = _load()
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(12)
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    return lib.synth_ray_value(_dptr(P), float(u), float(v), _dptr(prim), prim.shape[0])


def rigid_motion(n_views: int, rot_deg: float, trans_mm: float, rng: np.random.Generator) -> np.ndarray:
    """Per-view motion theta [n_views, 6] = (rx, ry, rz [rad], tx, ty, tz [mm]),
    rotations N(0, rot_deg) and translations N(0, trans_mm)."""
    th = np.zeros((n_views, 6))
    th[:, :3] = np.deg2rad(rot_deg) * rng.standard_normal((n_views, 3))
    th[:, 3:] = trans_mm * rng.standard_normal((n_views, 3))
    return th


def make_scan(cfg: ScanConfig, with_images: bool = True, views=None, n_threads: int | None = None) -> dict:
    """Everything one workload needs: P [N,3,4], images [N,H,W] FP32 (optional),
    the phantom, and the seeded motion (zeros if the config has none).
    ``views`` selects a subset of view indices (same phantom and trajectory)."""
    rng = np.random.Generator(np.random.PCG64(cfg.seed))
    prim = phantom(cfg, rng)
    P = trajectory(cfg)
    mrng = np.random.Generator(np.random.PCG64(cfg.seed + 7))
    motion = rigid_motion(cfg.n_views, cfg.motion_rot_deg, cfg.motion_trans_mm, mrng)
    if views is not None:
        views = np.asarray(views)
        P = P[views]
        motion = motion[views]
    out = {"cfg": cfg, "P": P, "prim": prim, "motion": motion}
    if with_images:
        out["images"] = project(P, prim, cfg.W, cfg.H, n_threads)
    return out


def upper_pairs(n_views: int) -> np.ndarray:
    """All unordered pairs a < b in row-major order, int32 [n_pairs, 2]."""
    a, b = np.triu_indices(n_views, k=1)
    return np.stack([a, b], axis=1).astype(np.int32)
