"""The library's per-view / per-pair FP64 set-up (the same __host__ __device__ code
the GPU kernels run), executed on the CPU through an internal host entry point and
checked against the oracle: sampled arc, step, N_kappa and the valid-sample set."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import oracle as orc
from paper_1806_02637_gb300 import build as ecc_build

_dp = ctypes.POINTER(ctypes.c_double)


def _lib():
    lib = ctypes.CDLL(ecc_build.build())
    f = lib.ecc_internal_setup_pair_host
    f.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  _dp, _dp]
    f.restype = ctypes.c_int
    return f


def _setup(P, motion, W, H, K, a, b):
    f = _lib()
    P = np.ascontiguousarray(P, dtype=np.float64)
    mot = None if motion is None else np.ascontiguousarray(motion, dtype=np.float64)
    info, A = np.zeros(8), np.zeros(12)
    rc = f(P.shape[0], P.ctypes.data_as(_dp), None if mot is None else mot.ctypes.data_as(_dp), W, H, K, a, b,
           info.ctypes.data_as(_dp), A.ctypes.data_as(_dp))
    assert rc == 0
    return info, A


def _valid_set(info, K):
    r0hi, r1lo, r1hi = int(info[5]), int(info[6]), int(info[7])
    v = np.zeros(K, bool)
    v[:r0hi] = True
    v[r1lo:r1hi] = True
    return v


CASES = [("c1", None, [(0, 1)], False),
         ("c2", tuple(range(0, 496, 31)), [(0, 1), (0, 15), (3, 9), (7, 8), (2, 14)], False),
         ("c3", tuple(range(0, 248, 17)), [(0, 1), (0, 14), (4, 11), (9, 10)], True),
         ("c4", (0, 1, 310, 619, 620, 930), [(0, 4), (0, 3), (1, 4), (2, 5), (0, 1), (3, 4)], False)]


@pytest.mark.parametrize("name,views,pairs,motion", CASES)
def test_host_setup_matches_oracle(name, views, pairs, motion):
    cfg = synth.CONFIGS[name]
    sc = synth.make_scan(cfg, with_images=False, views=None if views is None else np.array(views))
    P = sc["P"].reshape(-1, 12)
    th = sc["motion"] if motion else None
    K = cfg.K
    for a, b in pairs:
        info, A = _setup(P, th, cfg.W, cfg.H, K, a, b)
        arcs = orc.pair_arcs(P[a], P[b], cfg.W, cfg.H,
                             None if th is None else th[a], None if th is None else th[b])
        assert info[4] == 0
        # step of the sampled (shorter) arc
        assert np.isclose(info[2], arcs[2] / K, rtol=1e-12), (info[2], arcs[2] / K)
        # first sample direction = arc start rotated by half a step (mod pi)
        ang = np.arctan2(info[1], info[0]) - 0.5 * info[2]
        dlo = np.mod(ang - arcs[1] + 0.5 * np.pi, np.pi) - 0.5 * np.pi
        assert abs(dlo) < 1e-12, dlo
        # valid samples: membership of the sampled planes in the other view's arc
        kap = arcs[1] + (np.arange(K) + 0.5) * arcs[2] / K
        x = np.mod(kap - arcs[3], np.pi)
        want = x <= arcs[4]
        got = _valid_set(info, K)
        assert np.array_equal(got, want), (a, b, np.nonzero(got != want))
        assert int(info[3]) == int(want.sum())


def test_host_setup_degenerate_pair():
    cfg = synth.CONFIGS["c1"]
    sc = synth.make_scan(cfg, with_images=False)
    P = np.stack([sc["P"][0], 3.0 * sc["P"][0]]).reshape(-1, 12)
    info, _ = _setup(P, None, cfg.W, cfg.H, cfg.K, 0, 1)
    assert info[4] == 1 and info[3] == 0


@pytest.mark.parametrize("name,stride,n_pairs,seed", [("c2", 4, 400, 5), ("c3", 2, 300, 6), ("c4", 10, 400, 7)])
def test_host_setup_many_pairs(name, stride, n_pairs, seed):
    """Seeded random pairs of the scan: the sampled arc, step and valid-sample set of
    the (double-float) set-up against the oracle's FP64 arcs, pair by pair."""
    cfg = synth.CONFIGS[name]
    views = np.arange(0, cfg.n_views, stride)
    sc = synth.make_scan(cfg, with_images=False, views=views)
    P = sc["P"].reshape(-1, 12)
    th = sc["motion"] if cfg.motion_rot_deg > 0 else None
    rng = np.random.default_rng(seed)
    n = len(views)
    K = cfg.K
    for _ in range(n_pairs):
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        info, _ = _setup(P, th, cfg.W, cfg.H, K, a, b)
        arcs = orc.pair_arcs(P[a], P[b], cfg.W, cfg.H, None if th is None else th[a], None if th is None else th[b])
        assert info[4] == 0
        assert np.isclose(info[2], arcs[2] / K, rtol=1e-12)
        kap = arcs[1] + (np.arange(K) + 0.5) * arcs[2] / K
        want = np.mod(kap - arcs[3], np.pi) <= arcs[4]
        assert np.array_equal(_valid_set(info, K), want), (a, b)
