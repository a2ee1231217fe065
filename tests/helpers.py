"""Shared helpers of the parity tests: cached seeded workloads, oracle sinograms,
per-pair energies and the tolerance measures (test infrastructure)."""
from __future__ import annotations

import functools

import numpy as np

import synth
from oracle import oracle as orc

# FP32 paths must match the FP64 oracle within this relative error (per pair the
# denominator is max(d, FLOOR * E_ab), E_ab the mean of (S_a^2 + S_b^2)/2 over the
# pair's valid planes: d is a difference of nearly equal values for consistent
# pairs, and any FP32 arithmetic is only relative to E_ab there).
TOL_F32 = 1e-5
FLOOR = 1e-2


@functools.lru_cache(maxsize=None)
def scan(name: str, views: tuple | None = None):
    cfg = synth.CONFIGS[name]
    sc = synth.make_scan(cfg, views=None if views is None else np.array(views))
    return sc


@functools.lru_cache(maxsize=None)
def oracle_sino(name: str, views: tuple | None = None, n_alpha: int | None = None, n_s: int | None = None):
    cfg = synth.CONFIGS[name]
    sc = scan(name, views)
    return orc.radon_derivative(sc["P"], sc["images"], n_alpha or cfg.n_alpha, n_s or cfg.n_s)


def energies(P, sino, W, H, K, pairs, motion=None):
    """E_ab for each pair, from the oracle with zero-sinogram copies of the views."""
    P = np.asarray(P).reshape(-1, 3, 4)
    n = P.shape[0]
    P2 = np.concatenate([P, P])
    S2 = np.concatenate([sino, np.zeros_like(sino)])
    m2 = None if motion is None else np.concatenate([motion, motion])
    pairs = np.asarray(pairs)
    pa = np.stack([pairs[:, 0], pairs[:, 1] + n], axis=1)
    pb = np.stack([pairs[:, 0] + n, pairs[:, 1]], axis=1)
    ea = orc.ecc(P2, S2, W, H, K, motion=m2, pairs=pa)["d"]
    eb = orc.ecc(P2, S2, W, H, K, motion=m2, pairs=pb)["d"]
    return 0.5 * (ea + eb)


def pair_rel_err(d_gpu, d_ref, E):
    return np.abs(np.asarray(d_gpu) - np.asarray(d_ref)) / np.maximum(np.asarray(d_ref), FLOOR * np.asarray(E))


def sino_rel_err(S_gpu, S_ref):
    """Per view max|dS| / max|S|."""
    S_gpu = np.asarray(S_gpu, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    num = np.abs(S_gpu - S_ref).reshape(S_ref.shape[0], -1).max(axis=1)
    den = np.abs(S_ref).reshape(S_ref.shape[0], -1).max(axis=1)
    return num / den


def p_entry_scale(P):
    """Per-entry scale of projection matrices [n, 12]: the largest |M| entry of the
    row for the first three columns, |t| plus 100 times that for the last (a
    distance in mm times the row's scale).  Used to compare and step gradients with
    respect to P in units of relative change of each entry."""
    P = np.asarray(P, dtype=np.float64).reshape(-1, 3, 4)
    s = np.empty_like(P)
    s[:, :, :3] = np.abs(P[:, :, :3]).max(axis=2, keepdims=True)
    s[:, :, 3] = np.abs(P[:, :, 3]) + 100.0 * s[:, :, 0]
    return s.reshape(-1, 12)


def round_bf16(x):
    """Round to the nearest BF16 value (8 significant bits, ties to even), in FP64."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))   # x = m 2^e, 1/2 <= |m| < 1
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def quantize_f16(S):
    """FP16 storage with a per-view scale, as the precompute defines it: scale =
    max|S| / 2^14 of each view (FP32; 1 for an all-zero view), stored value =
    S / scale rounded to FP16.  Returns (stored FP16 array, FP32 scales)."""
    S = np.asarray(S, dtype=np.float64)
    amax = np.abs(S).reshape(S.shape[0], -1).max(axis=1).astype(np.float32)
    scales = np.where(amax > 0, amax / np.float32(16384.0), np.float32(1.0)).astype(np.float32)
    return (S / scales.astype(np.float64)[:, None, None]).astype(np.float16), scales
