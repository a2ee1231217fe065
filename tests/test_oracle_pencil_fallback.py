"""Pins of the pencil frame's fallback axis (reading R3 of the plane parametrisation
around the baseline, Eq. 13/14): when up_a + up_b is parallel to the baseline, the
world axis least aligned with the baseline replaces it.

The geometry that reaches it: two views at the same gantry angle whose sources are
shifted along the rotation axis (z).  Both detectors have the up axis (0, 0, -1),
the baseline is along z, and r - (r.u) u vanishes.

* the oracle's frame equals a numpy restatement of the rule, and is orthonormal
  with w and v normal to the baseline (every plane of the pencil contains it);
* the oracle's pair sum equals an independent numpy pair sum in that frame;
* its valid arcs equal a dense scan of the detector hit test.  The epipole lies at
  infinity along the detector columns here, so two corners share each corner line
  and two of the four gaps between corner angles have zero width (their midpoint
  lines graze an edge);
* with exact geometry and untruncated data the pair is consistent (Eq. 2) to the
  discretisation level, while data from a gantry turned by one more degree is not:
  a frame whose planes missed a source would break this.
"""
import functools

import numpy as np

import synth
from oracle import oracle as orc
from tests.test_oracle_ecc import _np_lookup, _np_view

CFG = synth.ScanConfig("fallback", n_views=2, arc_deg=90.0, full_scan=False, W=256, H=256, pixel_mm=1.0,
                       phantom="blobs", n_prim=3, size_range=(10.0, 20.0), value_range=(0.01, 0.02),
                       n_alpha=256, n_s=363, K=256, seed=4242)
THETA = np.deg2rad(30.0)
SHIFT = 2.0   # mm along z


def shifted_pair(shift=SHIFT, turn_deg=0.0):
    P0 = synth.projection_matrix(THETA, CFG.W, CFG.H, CFG.pixel_mm, CFG.sid, CFG.sdd)
    P1 = synth.projection_matrix(THETA + np.deg2rad(turn_deg), CFG.W, CFG.H, CFG.pixel_mm, CFG.sid, CFG.sdd)
    return np.stack([P0, orc.apply_motion(P1, [0.0, 0.0, 0.0, 0.0, 0.0, shift])])


@functools.lru_cache(maxsize=None)
def _data():
    prim = synth.phantom(CFG, np.random.default_rng(CFG.seed))
    P = shifted_pair()
    images = synth.project(P, prim, CFG.W, CFG.H)
    S = orc.radon_derivative(P, images, CFG.n_alpha, CFG.n_s)
    # view b's data as a gantry turned by a further 1 degree would record it (a shift
    # along the baseline itself leaves every plane of the pencil unchanged, so it is
    # no negative control), evaluated with the unturned geometry
    Pw = shifted_pair(turn_deg=1.0)
    S_wrong = orc.radon_derivative(Pw, synth.project(Pw, prim, CFG.W, CFG.H), CFG.n_alpha, CFG.n_s)
    return P, S, S_wrong


def np_fallback_frame(Pa, Pb):
    """The rule restated: u = baseline direction; the first axis whose |u_i| is within
    1e-9 of the smallest, minus its projection on u, normalised, is w; v = w x u."""
    _, _, Ca, _ = _np_view(Pa)
    _, _, Cb, _ = _np_view(Pb)
    u = (Cb - Ca) / np.linalg.norm(Cb - Ca)
    ax = int(np.nonzero(np.abs(u) <= np.abs(u).min() + 1e-9)[0][0])
    e = np.zeros(3)
    e[ax] = 1.0
    w = e - u[ax] * u
    w /= np.linalg.norm(w)
    return u, w, np.cross(w, u)


def test_geometry_reaches_the_fallback():
    P = shifted_pair()
    _, _, Ca, upa = _np_view(P[0])
    _, _, Cb, upb = _np_view(P[1])
    u = (Cb - Ca) / np.linalg.norm(Cb - Ca)
    r = upa + upb
    assert np.linalg.norm(r - (r @ u) * u) < 1e-6          # the regular construction is degenerate
    assert np.allclose(np.abs(u), [0.0, 0.0, 1.0], atol=1e-12)


def test_fallback_frame_matches_numpy_rule():
    P = shifted_pair()
    w, v = orc.pair_frame(P[0], P[1])
    u, w_np, v_np = np_fallback_frame(P[0], P[1])
    assert np.allclose(w, w_np, atol=1e-12) and np.allclose(v, v_np, atol=1e-12)
    assert abs(w @ u) < 1e-12 and abs(v @ u) < 1e-12 and abs(w @ v) < 1e-12
    assert np.isclose(np.linalg.norm(w), 1.0, atol=1e-12) and np.isclose(np.linalg.norm(v), 1.0, atol=1e-12)


def test_fallback_pair_sum_matches_independent_numpy():
    P, S, _ = _data()
    r = orc.ecc(P, S, CFG.W, CFG.H, CFG.K)
    lo, length = r["arcs"][0, 1], r["arcs"][0, 2]
    Pa, Ma, _, _ = _np_view(P[0])
    Pb, Mb, _, _ = _np_view(P[1])
    _, w, v = np_fallback_frame(P[0], P[1])
    kap = lo + (np.arange(CFG.K) + 0.5) * length / CFG.K
    n = np.cos(kap)[:, None] * w + np.sin(kap)[:, None] * v
    Sa, ha = _np_lookup(S[0], CFG.W, CFG.H, n @ (np.linalg.det(Ma) * np.linalg.inv(Ma)))
    Sb, hb = _np_lookup(S[1], CFG.W, CFG.H, n @ (np.linalg.det(Mb) * np.linalg.inv(Mb)))
    ok = ha & hb
    assert ok.sum() == r["nk"][0] > CFG.K // 2
    d = ((Sa - Sb) ** 2)[ok].sum() / ok.sum()
    assert np.isclose(d, r["d"][0], rtol=1e-10)


def test_fallback_pair_consistent_with_exact_geometry():
    P, S, S_wrong = _data()
    d = orc.ecc(P, S, CFG.W, CFG.H, CFG.K)["d"][0]
    zero = S.copy()
    zero[1] = 0.0
    energy = orc.ecc(P, zero, CFG.W, CFG.H, CFG.K)["d"][0]
    assert d <= 1e-5 * energy, (d, energy)
    mixed = np.stack([S[0], S_wrong[1]])
    d_wrong = orc.ecc(P, mixed, CFG.W, CFG.H, CFG.K)["d"][0]
    assert d_wrong > 100.0 * d, (d_wrong, d)


def test_fallback_arcs_match_dense_hit_scan():
    P = shifted_pair()
    arcs = orc.pair_arcs(P[0], P[1], CFG.W, CFG.H)
    _, w, v = np_fallback_frame(P[0], P[1])
    n_dense = 40000
    kap = -np.pi / 2 + (np.arange(n_dense) + 0.5) * np.pi / n_dense
    nn = np.cos(kap)[:, None] * w + np.sin(kap)[:, None] * v
    sampled = int(arcs[0])
    for view, lo, length in ((sampled, arcs[1], arcs[2]), (1 - sampled, arcs[3], arcs[4])):
        _, M, _, _ = _np_view(P[view])
        _, hit = _np_lookup(np.zeros((4, 8)), CFG.W, CFG.H, nn @ (np.linalg.det(M) * np.linalg.inv(M)))
        x = np.mod(kap - lo, np.pi)
        inside = x <= length
        edge = (np.abs(x) < 1e-4) | (np.abs(x - length) < 1e-4) | (np.abs(x - np.pi) < 1e-4)
        assert 0.0 < length < np.pi
        assert np.array_equal(inside[~edge], hit[~edge])
