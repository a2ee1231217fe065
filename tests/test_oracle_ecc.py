"""Pins of the oracle's consistency metric (Eq. 15-17): an independent numpy
re-implementation of one pair's sum (cofactor lines, own bilinear look-up), the
arcs against a dense scan of the detector hit test, and the invariants the
geometry fixes (exact data, pair symmetry, scaling of P, global rigid motion,
detectability of out-of-plane motion)."""
import functools

import numpy as np
import pytest

import synth
from oracle import oracle as orc


@functools.lru_cache(maxsize=None)
def _c1():
    cfg = synth.CONFIGS["c1"]
    sc = synth.make_scan(cfg)
    S = orc.radon_derivative(sc["P"], sc["images"], cfg.n_alpha, cfg.n_s)
    return cfg, sc, S


@functools.lru_cache(maxsize=None)
def _c2_subset():
    """Eight views of the 496-view short scan (every 62nd), reduced sinogram grid."""
    cfg = synth.CONFIGS["c2"]
    sc = synth.make_scan(cfg, views=np.arange(0, 496, 62))
    S = orc.radon_derivative(sc["P"], sc["images"], 192, 256)
    return cfg, sc, S


# ----------------------------------------------------------- independent re-implementation
def _np_view(P):
    P = np.asarray(P, float).reshape(3, 4)
    M = P[:, :3]
    P = P / np.linalg.norm(M[2]) * np.sign(np.linalg.det(M))
    M = P[:, :3]
    C = -np.linalg.solve(M, P[:, 3])
    up = np.cross(M[2], M[0])
    return P, M, C, up / np.linalg.norm(up)


def _np_lookup(sino, W, H, l):
    """Vectorised look-up, written independently of the oracle's C code."""
    n_alpha, n_s = sino.shape
    cx, cy = (W - 1) / 2, (H - 1) / 2
    l = np.atleast_2d(l)
    h = np.hypot(l[:, 0], l[:, 1])
    c, s_ = l[:, 0] / h, l[:, 1] / h
    s = -(l[:, 2] + l[:, 0] * cx + l[:, 1] * cy) / h
    hit = np.abs(s) <= W / 2 * np.abs(c) + H / 2 * np.abs(s_)
    alpha = np.arctan2(s_, c)
    sign = np.where(alpha < 0, -1.0, 1.0)
    s = np.where(alpha < 0, -s, s)
    alpha = np.where(alpha < 0, alpha + np.pi, alpha)
    # alpha = pi (a line with l2 = +0 and l1 < 0, or -tiny + pi rounding up) folds to 0
    top = alpha >= np.pi
    sign = np.where(top, -sign, sign)
    s = np.where(top, -s, s)
    alpha = np.where(top, alpha - np.pi, alpha)
    ia = alpha * n_alpha / np.pi
    is_ = s / (np.hypot(W, H) / (n_s - 1)) + (n_s - 1) / 2
    # extend the sinogram by the wrapped row: row n_alpha = -row 0 mirrored in s
    ext = np.vstack([sino, -sino[0, ::-1][None]])
    ext = np.pad(ext, ((0, 0), (2, 2)))
    m0 = np.floor(ia).astype(int)
    n0 = np.floor(is_).astype(int)
    fa, fs = ia - m0, is_ - n0
    n0c = np.clip(n0 + 2, 0, n_s + 2)
    n1c = np.clip(n0 + 3, 0, n_s + 3)
    val = ((1 - fa) * ((1 - fs) * ext[m0, n0c] + fs * ext[m0, n1c])
           + fa * ((1 - fs) * ext[m0 + 1, n0c] + fs * ext[m0 + 1, n1c]))
    return sign * val, hit


def _np_pair(Pa, Pb, sa, sb, W, H, K, lo, length):
    Pa, Ma, Ca, upa = _np_view(Pa)
    Pb, Mb, Cb, upb = _np_view(Pb)
    u = (Cb - Ca) / np.linalg.norm(Cb - Ca)
    r = upa + upb
    w = r - (r @ u) * u
    w /= np.linalg.norm(w)
    v = np.cross(w, u)
    kap = lo + (np.arange(K) + 0.5) * length / K
    n = np.cos(kap)[:, None] * w + np.sin(kap)[:, None] * v
    cofa = np.linalg.det(Ma) * np.linalg.inv(Ma).T
    cofb = np.linalg.det(Mb) * np.linalg.inv(Mb).T
    Sa, ha = _np_lookup(sa, W, H, n @ cofa.T)
    Sb, hb = _np_lookup(sb, W, H, n @ cofb.T)
    ok = ha & hb
    return ((Sa - Sb) ** 2)[ok].sum() / max(ok.sum(), 1), int(ok.sum())


def test_pair_sum_matches_independent_numpy():
    cfg, sc, S = _c1()
    th = np.zeros((2, 6))
    th[1] = [0.01, -0.004, 0.02, 0.5, -1.0, 1.5]
    r = orc.ecc(sc["P"], S, cfg.W, cfg.H, cfg.K, motion=th)
    Pm = [orc.apply_motion(sc["P"][i], th[i]) for i in range(2)]
    lo, length = r["arcs"][0, 1], r["arcs"][0, 2]
    d, nk = _np_pair(Pm[0], Pm[1], S[0], S[1], cfg.W, cfg.H, cfg.K, lo, length)
    assert nk == r["nk"][0]
    assert np.isclose(d, r["d"][0], rtol=1e-10)


def test_pair_sum_matches_independent_numpy_short_scan():
    cfg, sc, S = _c2_subset()
    r = orc.ecc(sc["P"], S, cfg.W, cfg.H, 96, pairs=[[0, 3], [2, 7], [1, 2]])
    for p, (a, b) in enumerate(r["pairs"]):
        d, nk = _np_pair(sc["P"][a], sc["P"][b], S[a], S[b], cfg.W, cfg.H, 96, r["arcs"][p, 1], r["arcs"][p, 2])
        assert nk == r["nk"][p]
        assert np.isclose(d, r["d"][p], rtol=1e-10)


def _dense_valid(Pa, Pb, W, H, view, n=40000):
    """Brute-force valid set of pencil angles for one view by the hit test."""
    Pa_, Ma, Ca, upa = _np_view(Pa)
    Pb_, Mb, Cb, upb = _np_view(Pb)
    u = (Cb - Ca) / np.linalg.norm(Cb - Ca)
    r = upa + upb
    w = r - (r @ u) * u
    w /= np.linalg.norm(w)
    v = np.cross(w, u)
    kap = -np.pi / 2 + (np.arange(n) + 0.5) * np.pi / n
    nn = np.cos(kap)[:, None] * w + np.sin(kap)[:, None] * v
    M = Ma if view == 0 else Mb
    cof = np.linalg.det(M) * np.linalg.inv(M).T
    l = nn @ cof.T
    _, hit = _np_lookup(np.zeros((4, 8)), W, H, l)
    return kap, hit


@pytest.mark.parametrize("pair", [(0, 1), (0, 4), (1, 6), (0, 7), (3, 5)])
def test_arcs_match_dense_hit_scan(pair):
    cfg, sc, S = _c2_subset()
    a, b = pair
    arcs = orc.pair_arcs(sc["P"][a], sc["P"][b], cfg.W, cfg.H)
    sampled = int(arcs[0])
    for view, lo, length in ((sampled, arcs[1], arcs[2]), (1 - sampled, arcs[3], arcs[4])):
        kap, hit = _dense_valid(sc["P"][a], sc["P"][b], cfg.W, cfg.H, view)
        x = np.mod(kap - lo, np.pi)
        inside = x <= length
        edge = (np.abs(x) < 1e-4) | (np.abs(x - length) < 1e-4) | (np.abs(x - np.pi) < 1e-4)
        assert np.array_equal(inside[~edge], hit[~edge])
    assert arcs[2] <= arcs[4]


def test_validity_tests_agree():
    """Membership in the other view's arc equals the detector hit test on every sample."""
    cfg, sc, S = _c2_subset()
    r = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128)
    assert r["mismatch"].sum() == 0
    assert (r["nk"] > 0).all() and (r["nk"] <= 128).all()


def test_exact_geometry_consistent():
    """Eq. (2): with exact geometry and untruncated data, d is at the discretisation level."""
    cfg, sc, S = _c1()
    r = orc.ecc(sc["P"], S, cfg.W, cfg.H, cfg.K)
    zero = S.copy()
    zero[1] = 0.0
    energy = orc.ecc(sc["P"], zero, cfg.W, cfg.H, cfg.K)["d"][0]   # mean S_a^2 over valid planes
    assert r["d"][0] <= 1e-6 * energy
    th = np.zeros((2, 6))
    th[1, 5] = 1.0
    moved = orc.ecc(sc["P"], S, cfg.W, cfg.H, cfg.K, motion=th)["d"][0]
    assert moved > 1e3 * r["d"][0]


def test_pair_symmetry():
    cfg, sc, S = _c2_subset()
    r1 = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128, pairs=[[0, 3], [2, 6], [1, 7]])
    r2 = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128, pairs=[[3, 0], [6, 2], [7, 1]])
    assert np.array_equal(r1["nk"], r2["nk"])
    assert np.allclose(r1["d"], r2["d"], rtol=1e-10)


@pytest.mark.parametrize("sigma", [-3.0, 0.5, 1e3])
def test_projection_scale_invariance(sigma):
    cfg, sc, S = _c2_subset()
    scale = np.ones(len(sc["P"]))
    scale[::2] = sigma
    r1 = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128)
    r2 = orc.ecc(sc["P"] * scale[:, None, None], S, cfg.W, cfg.H, 128)
    assert np.array_equal(r1["nk"], r2["nk"])
    assert np.allclose(r1["d"], r2["d"], rtol=1e-9)


def test_global_rigid_motion_invariance():
    """The same T for every view moves the whole geometry rigidly: nothing changes."""
    cfg, sc, S = _c2_subset()
    th = np.tile([0.03, -0.05, 0.2, 4.0, -3.0, 6.0], (len(sc["P"]), 1))
    r1 = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128)
    r2 = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128, motion=th)
    assert np.array_equal(r1["nk"], r2["nk"])
    assert np.allclose(r1["d"], r2["d"], rtol=1e-8)


def test_out_of_plane_motion_detected():
    """Out-of-plane (z) translation raises the total strongly; rotation about the
    trajectory axis (motion along the mostly horizontal epipolar lines) barely does
    (the detectability remark of the Experiments section)."""
    cfg, sc, S = _c2_subset()
    nv = len(sc["P"])
    base = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128)["total"]
    rng = np.random.default_rng(11)
    tz = np.zeros((nv, 6))
    tz[:, 5] = rng.normal(0, 2.0, nv)
    rz = np.zeros((nv, 6))
    rz[:, 2] = rng.normal(0, np.deg2rad(1.0), nv)
    t_tz = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128, motion=tz)["total"]
    t_rz = orc.ecc(sc["P"], S, cfg.W, cfg.H, 128, motion=rz)["total"]
    assert t_tz > 100 * base
    assert t_rz < 0.05 * t_tz


def test_pinv_construction_same_result():
    """The paper's claim: both line constructions produce the same results."""
    cfg, sc, S = _c1()
    th = np.zeros((2, 6))
    th[1, 5] = 1.0
    r1 = orc.ecc(sc["P"], S, cfg.W, cfg.H, cfg.K, motion=th)
    r2 = orc.ecc(sc["P"], S, cfg.W, cfg.H, cfg.K, motion=th, construction="pinv")
    assert np.array_equal(r1["nk"], r2["nk"])
    assert np.allclose(r1["d"], r2["d"], rtol=1e-6)


def test_cauchy_norm():
    """Eq. (16): e = d / (1 + d/c); c <= 0 disables it; e -> d as c grows."""
    cfg, sc, S = _c2_subset()
    r0 = orc.ecc(sc["P"], S, cfg.W, cfg.H, 64)
    c = float(np.median(r0["d"]))
    r1 = orc.ecc(sc["P"], S, cfg.W, cfg.H, 64, cauchy_c=c)
    assert np.allclose(r1["e"], r0["d"] / (1 + r0["d"] / c), rtol=1e-14)
    assert np.allclose(r0["e"], r0["d"])
    r2 = orc.ecc(sc["P"], S, cfg.W, cfg.H, 64, cauchy_c=1e12 * c)
    assert np.allclose(r2["e"], r0["d"], rtol=1e-9)
    assert np.isclose(r1["total"], r1["e"].sum(), rtol=1e-14)
