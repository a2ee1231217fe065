"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs: sinograms (Eq. 1), per-pair d, e, N_kappa and totals (Eq. 15-17),
edge cases, and full-size launches checked on sampled pairs."""
import functools

import numpy as np
import pytest

import synth
from oracle import oracle as orc
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@functools.lru_cache(maxsize=None)
def _ctx():
    import paper_1806_02637_gb300 as ecc
    return ecc.Context(0)


def _ecc():
    import paper_1806_02637_gb300 as ecc
    return ecc


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _gpu_sino(sc, n_alpha, n_s, dtype=None):
    ecc = _ecc()
    S, scales = ecc.ecc_precompute_radon_derivative(_ctx(), _cuda(sc["P"]), _cuda(sc["images"]), n_alpha, n_s,
                                                    dtype=dtype)
    torch.cuda.synchronize()
    return S, scales


def _gpu_eval(P, S_t, W, Hh, K, c=0.0, motion=None, pairs=None, scales=None):
    ecc = _ecc()
    r = ecc.ecc_evaluate(_ctx(), _cuda(P), S_t, W, Hh, K, cauchy_c=c,
                         motion=None if motion is None else _cuda(motion),
                         pairs=None if pairs is None else _cuda(np.asarray(pairs, dtype=np.int32)), scales=scales)
    torch.cuda.synchronize()
    return (float(r["total"].cpu()[0]), r["per_pair"].cpu().numpy(), r["nkappa"].cpu().numpy())


# ----------------------------------------------------------------- sinograms
@pytest.mark.parametrize("name,views", [("c1", None), ("c2", (0, 97, 250, 311, 495)), ("c3", (5, 200))])
def test_radon_parity(name, views):
    cfg = synth.CONFIGS[name]
    sc = H.scan(name, views)
    S, _ = _gpu_sino(sc, cfg.n_alpha, cfg.n_s)
    ref = H.oracle_sino(name, views)
    err = H.sino_rel_err(S.cpu().numpy(), ref)
    assert err.max() <= H.TOL_F32, err


def test_radon_parity_large_detector_ragged_grid():
    """976^2 detector, 1024 x 1382 grid (n_s not a multiple of the 31-wide chunks)."""
    cfg = synth.CONFIGS["c4"]
    sc = H.scan("c4", (7,))
    S, _ = _gpu_sino(sc, cfg.n_alpha, cfg.n_s)
    ref = H.oracle_sino("c4", (7,))
    assert H.sino_rel_err(S.cpu().numpy(), ref).max() <= H.TOL_F32


@pytest.mark.parametrize("n_alpha,n_s", [(4, 2), (5, 3), (37, 61), (180, 129)])
def test_radon_parity_small_grids(n_alpha, n_s):
    sc = H.scan("c1")
    S, _ = _gpu_sino(sc, n_alpha, n_s)
    ref = orc.radon_derivative(sc["P"], sc["images"], n_alpha, n_s)
    assert H.sino_rel_err(S.cpu().numpy(), ref).max() <= H.TOL_F32


# --------------------------------------------------------------- ECC (Eq. 15-17)
def _check_pairs(P, S32, W, Hh, K, c=0.0, motion=None, pairs=None):
    """GPU vs oracle on the same FP32 sinogram values."""
    total, pp, nk = _gpu_eval(P, _cuda(S32), W, Hh, K, c, motion, pairs)
    ref = orc.ecc(P, S32.astype(np.float64), W, Hh, K, cauchy_c=c, motion=motion, pairs=pairs)
    assert np.array_equal(nk, ref["nk"]), np.nonzero(nk != ref["nk"])
    E = H.energies(P, S32.astype(np.float64), W, Hh, K, ref["pairs"], motion)
    err_d = H.pair_rel_err(pp[:, 0], ref["d"], E)
    err_e = H.pair_rel_err(pp[:, 1], ref["e"], E)
    assert err_d.max() <= H.TOL_F32, (err_d.max(), np.argmax(err_d))
    assert err_e.max() <= H.TOL_F32
    # the total uses the same floor, summed over the pairs (plain relative error
    # whenever the pairs are inconsistent beyond FLOOR * E_ab)
    assert abs(total - ref["total"]) <= H.TOL_F32 * np.maximum(ref["e"], H.FLOOR * E).sum()
    return total, pp, nk, ref


def test_ecc_parity_c1_exact_and_moved():
    cfg = synth.CONFIGS["c1"]
    sc = H.scan("c1")
    S32 = H.oracle_sino("c1").astype(np.float32)
    _check_pairs(sc["P"], S32, cfg.W, cfg.H, cfg.K)
    th = np.zeros((2, 6))
    th[1] = [0.01, -0.004, 0.02, 0.5, -1.0, 1.5]
    _check_pairs(sc["P"], S32, cfg.W, cfg.H, cfg.K, c=1e-3, motion=th)


def test_ecc_parity_maximum_kappa():
    """n_kappa at the API maximum (65536 planes, 2048 tiles) on the two-view scan."""
    cfg = synth.CONFIGS["c1"]
    sc = H.scan("c1")
    S32 = H.oracle_sino("c1").astype(np.float32)
    _check_pairs(sc["P"], S32, cfg.W, cfg.H, 65536)


SUB = tuple(range(0, 496, 21))  # 24 views of the 496-view short scan


@pytest.mark.parametrize("K", [512, 77, 1024, 1])
def test_ecc_parity_short_scan_subset(K):
    cfg = synth.CONFIGS["c2"]
    sc = H.scan("c2", SUB)
    S32 = H.oracle_sino("c2", SUB).astype(np.float32)
    _check_pairs(sc["P"], S32, cfg.W, cfg.H, K)


def test_ecc_parity_motion_cauchy_pair_list():
    cfg = synth.CONFIGS["c3"]
    views = tuple(range(0, 248, 11))
    sc = H.scan("c3", views)
    S32 = H.oracle_sino("c3", views).astype(np.float32)
    rng = np.random.default_rng(3)
    n = len(views)
    pairs = np.array([(a, b) for a in range(n) for b in range(n) if a != b])[rng.choice(n * (n - 1), 150, False)]
    _, pp, _, ref = _check_pairs(sc["P"], S32, cfg.W, cfg.H, cfg.K, c=0.0, motion=sc["motion"], pairs=pairs)
    c = float(np.median(ref["d"]))
    _check_pairs(sc["P"], S32, cfg.W, cfg.H, cfg.K, c=c, motion=sc["motion"], pairs=pairs)


@functools.lru_cache(maxsize=None)
def _opposed_case():
    views = (0, 1, 310, 619, 620, 621, 930, 1239)
    sc = H.scan("c4", views)
    return sc, orc.radon_derivative(sc["P"], sc["images"], 256, 346).astype(np.float32)


# The evaluation takes tiles of 64 samples; the last one holds K mod 64 (or 64): 36 and 33
# (33..63: anchored at the mean of its two 32-sample centres), 32 and 13 (at most 32: its
# own centre), 63 (a single ragged tile), 64 (no ragged tile), 1.
@pytest.mark.parametrize("K", [256, 77, 100, 97, 96, 64, 63, 33, 1])
def test_ecc_full_scan_with_opposed_views(K):
    """Full 360-degree geometry: opposed views take the full-pi arc branch (tiles cross
    the alpha fold); K not a multiple of 64 adds a ragged last tile."""
    cfg = synth.CONFIGS["c4"]
    sc, S32 = _opposed_case()
    _, _, nk, ref = _check_pairs(sc["P"], S32, cfg.W, cfg.H, K)
    full = ref["arcs"][:, 2] > 3.14
    assert full.any()


@pytest.mark.parametrize("K", [512, 100, 77])
def test_two_pairs_per_warp_equal_one_pair_per_warp(K):
    """A launch of at least three waves of 16-pair blocks (all 30,628 pairs of the
    248-view scan) gives each warp two pairs; an explicit list of 4,000 of them gives
    each warp one.  Every pair's anchors and sums are the same code either way, so
    d, e and N_kappa agree bitwise."""
    cfg = synth.CONFIGS["c3"]
    sc = H.scan("c3")
    n = len(sc["P"])
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    if n * (n - 1) // 2 < 3 * 16 * 4 * n_sm:
        pytest.skip("this GPU needs more pairs for two pairs per warp")
    S, _ = _gpu_sino(sc, cfg.n_alpha, cfg.n_s)
    _, pp, nk = _gpu_eval(sc["P"], S, cfg.W, cfg.H, K)
    sel = np.sort(np.random.default_rng(K).choice(n * (n - 1) // 2, 4000, replace=False))
    _, pp1, nk1 = _gpu_eval(sc["P"], S, cfg.W, cfg.H, K, pairs=synth.upper_pairs(n)[sel])
    assert np.array_equal(nk[sel], nk1)
    assert np.array_equal(pp[sel], pp1)


def test_full_size_launch_sampled_pairs():
    """All 122,760 pairs of the 496-view scan in one launch (the benchmark's
    configuration); pairs among 40 sampled views are compared with the oracle on
    oracle sinograms, the rest run on GPU-computed sinograms."""
    cfg = synth.CONFIGS["c2"]
    full = H.scan("c2")
    views = tuple(int(v) for v in np.random.default_rng(496).choice(496, 40, replace=False))
    S_all, _ = _gpu_sino(full, cfg.n_alpha, cfg.n_s)
    S_or = H.oracle_sino("c2", tuple(sorted(views))).astype(np.float32)
    idx = torch.tensor(sorted(views), device="cuda")
    # the full-size precompute (batched launches) on the sampled views
    assert H.sino_rel_err(S_all[idx].cpu().numpy(), S_or).max() <= H.TOL_F32
    S_all[idx] = _cuda(S_or)
    total, pp, nk = _gpu_eval(full["P"], S_all, cfg.W, cfg.H, cfg.K)
    sv = np.array(sorted(views))
    sub_pairs = np.array([(i, j) for i in range(40) for j in range(i + 1, 40)])
    ga, gb = sv[sub_pairs[:, 0]], sv[sub_pairs[:, 1]]
    n = 496
    flat = ga * (2 * n - ga - 1) // 2 + (gb - ga - 1)
    ref = orc.ecc(full["P"][sv], S_or.astype(np.float64), cfg.W, cfg.H, cfg.K, pairs=sub_pairs)
    assert np.array_equal(nk[flat], ref["nk"])
    E = H.energies(full["P"][sv], S_or.astype(np.float64), cfg.W, cfg.H, cfg.K, sub_pairs)
    err = H.pair_rel_err(pp[flat, 0], ref["d"], E)
    assert err.max() <= H.TOL_F32, err.max()
    assert np.isfinite(pp).all() and (nk > 0).all() and (nk <= cfg.K).all()
    assert np.isclose(total, pp[:, 1].sum(), rtol=1e-9)


# ------------------------------------------------------------------ end to end
def test_end_to_end_c1():
    """Images -> sinograms -> total, both sides from the same images."""
    cfg = synth.CONFIGS["c1"]
    sc = H.scan("c1")
    S, _ = _gpu_sino(sc, cfg.n_alpha, cfg.n_s)
    th = np.zeros((2, 6))
    th[1, 5] = 1.0
    total, pp, nk = _gpu_eval(sc["P"], S, cfg.W, cfg.H, cfg.K, motion=th)
    ref = orc.ecc(sc["P"], H.oracle_sino("c1"), cfg.W, cfg.H, cfg.K, motion=th)
    assert np.array_equal(nk, ref["nk"])
    assert abs(total - ref["total"]) <= H.TOL_F32 * ref["total"]


def test_host_entry_matches_device_path():
    ecc = _ecc()
    cfg = synth.CONFIGS["c2"]
    sc = H.scan("c2", SUB)
    t_host = ecc.ecc_scan_consistency_host(_ctx(), sc["P"], sc["images"], cfg.n_alpha, cfg.n_s, cfg.K)
    S, _ = _gpu_sino(sc, cfg.n_alpha, cfg.n_s)
    t_dev, _, _ = _gpu_eval(sc["P"], S, cfg.W, cfg.H, cfg.K)
    assert t_host == t_dev
    ref = orc.ecc(sc["P"], H.oracle_sino("c2", SUB), cfg.W, cfg.H, cfg.K)["total"]
    assert abs(t_host - ref) <= H.TOL_F32 * ref


def test_host_entry_pinned_upload_in_batches():
    """From pinned host memory the images go up per precompute batch (47 views of c2's
    size per batch: three here) on a second stream, overlapping the projections.  The
    total equals the pageable call's and the device path's bitwise, call after call."""
    ecc = _ecc()
    cfg = synth.CONFIGS["c2"]
    views = tuple(range(0, 496, 5))[:100]
    sc = H.scan("c2", views)
    pinned = torch.from_numpy(np.ascontiguousarray(sc["images"], dtype=np.float32)).pin_memory()
    t_pinned = [ecc.ecc_scan_consistency_host(_ctx(), sc["P"], pinned, cfg.n_alpha, cfg.n_s, cfg.K) for _ in range(2)]
    t_pageable = ecc.ecc_scan_consistency_host(_ctx(), sc["P"], sc["images"], cfg.n_alpha, cfg.n_s, cfg.K)
    S, _ = _gpu_sino(sc, cfg.n_alpha, cfg.n_s)
    t_dev, _, _ = _gpu_eval(sc["P"], S, cfg.W, cfg.H, cfg.K)
    assert t_pinned[0] == t_pinned[1] == t_pageable == t_dev


def test_deterministic_and_pair_order():
    cfg = synth.CONFIGS["c2"]
    sc = H.scan("c2", SUB)
    S32 = _cuda(H.oracle_sino("c2", SUB).astype(np.float32))
    t1, p1, n1 = _gpu_eval(sc["P"], S32, cfg.W, cfg.H, cfg.K)
    t2, p2, n2 = _gpu_eval(sc["P"], S32, cfg.W, cfg.H, cfg.K)
    assert t1 == t2 and np.array_equal(p1, p2) and np.array_equal(n1, n2)
    pairs = synth.upper_pairs(len(SUB))
    t3, p3, n3 = _gpu_eval(sc["P"], S32, cfg.W, cfg.H, cfg.K, pairs=pairs)
    assert np.array_equal(p1, p3) and np.array_equal(n1, n3)
    # swapped pairs (b, a): same d up to the FP32 evaluation (the pencil is mirrored)
    t4, p4, n4 = _gpu_eval(sc["P"], S32, cfg.W, cfg.H, cfg.K, pairs=pairs[:, ::-1].copy())
    assert np.array_equal(n1, n4)
    assert np.allclose(p1[:, 0], p4[:, 0], rtol=1e-4, atol=1e-6 * p1[:, 0].max())


# ------------------------------------------------------------------ edge cases
def test_degenerate_pair_and_status():
    ecc = _ecc()
    cfg = synth.CONFIGS["c1"]
    sc = H.scan("c1")
    P = np.stack([sc["P"][0], sc["P"][0] * 2.0, sc["P"][1]])   # views 0 and 1 share a source
    S32 = np.concatenate([H.oracle_sino("c1")[:1], H.oracle_sino("c1")]).astype(np.float32)
    ecc.ecc_status(_ctx())
    total, pp, nk = _gpu_eval(P, _cuda(S32), cfg.W, cfg.H, cfg.K)
    assert nk[0] == 0 and pp[0, 0] == 0.0
    assert ecc.ecc_status(_ctx()) & 2
    assert ecc.ecc_status(_ctx()) == 0
    ref = orc.ecc(P[[0, 2]], S32[[0, 2]].astype(np.float64), cfg.W, cfg.H, cfg.K)
    assert nk[1] == ref["nk"][0]


def test_empty_pairs_and_invalid_arguments():
    ecc = _ecc()
    cfg = synth.CONFIGS["c1"]
    sc = H.scan("c1")
    S32 = _cuda(H.oracle_sino("c1").astype(np.float32))
    r = ecc.ecc_evaluate(_ctx(), _cuda(sc["P"]), S32, cfg.W, cfg.H, cfg.K,
                         pairs=torch.zeros((0, 2), dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    assert float(r["total"].cpu()[0]) == 0.0
    with pytest.raises(ecc.EccError):
        ecc.ecc_evaluate(_ctx(), _cuda(sc["P"]), S32, cfg.W, cfg.H, 0)
    with pytest.raises(ecc.EccError):
        ecc.ecc_evaluate(_ctx(), _cuda(sc["P"]), S32, 1, cfg.H, cfg.K)
    # the context stays usable
    total, _, _ = _gpu_eval(sc["P"], S32, cfg.W, cfg.H, cfg.K)
    assert np.isfinite(total)


def test_tiny_detector():
    """5 x 7 detector, 8 x 9 grid: every tile and chunk is ragged."""
    cfg = synth.ScanConfig("tiny", n_views=3, arc_deg=120.0, full_scan=False, W=7, H=5, pixel_mm=40.0,
                           phantom="blobs", n_prim=1, size_range=(8.0, 10.0), value_range=(0.01, 0.02),
                           n_alpha=8, n_s=9, K=40, seed=5)
    sc = synth.make_scan(cfg)
    S, _ = _gpu_sino(sc, cfg.n_alpha, cfg.n_s)
    ref = orc.radon_derivative(sc["P"], sc["images"], cfg.n_alpha, cfg.n_s)
    assert H.sino_rel_err(S.cpu().numpy(), ref).max() <= H.TOL_F32
    _check_pairs(sc["P"], ref.astype(np.float32), cfg.W, cfg.H, cfg.K)


def test_pencil_frame_fallback_pair():
    """Two views at one gantry angle with sources 2 mm apart along the rotation axis: the
    detectors' up axes sum to a vector along the baseline, so the pencil frame takes its
    fallback axis (reading R3), and the epipole lies at infinity along the detector
    columns.  The value, N_kappa and the motion gradient match the oracle."""
    from tests import test_oracle_pencil_fallback as F
    ecc = _ecc()
    P, S, _ = F._data()
    S32 = S.astype(np.float32)
    total, pp, nk = _gpu_eval(P, _cuda(S32), F.CFG.W, F.CFG.H, F.CFG.K)
    ref = orc.ecc(P, S32.astype(np.float64), F.CFG.W, F.CFG.H, F.CFG.K)
    assert np.array_equal(nk, ref["nk"]) and nk[0] > F.CFG.K // 2
    E = H.energies(P, S32.astype(np.float64), F.CFG.W, F.CFG.H, F.CFG.K, ref["pairs"])
    assert H.pair_rel_err(pp[:, 0], ref["d"], E).max() <= H.TOL_F32
    # the gradient at the fallback point (theta = 0), through the fallback axis's adjoint,
    # on inconsistent data (view b from a gantry turned by one more degree): nonzero
    _, S, S_wrong = F._data()
    Sm = np.stack([S[0], S_wrong[1]]).astype(np.float32)
    th = np.zeros((2, 6))
    r = ecc.ecc_evaluate_grad(_ctx(), _cuda(P), _cuda(Sm), F.CFG.W, F.CFG.H, F.CFG.K, motion=_cuda(th))
    torch.cuda.synchronize()
    g = r["grad"].cpu().numpy()
    gref = orc.ecc_grad(P, Sm.astype(np.float64), F.CFG.W, F.CFG.H, F.CFG.K, motion=th)["grad"]
    err = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    print(f"fallback pair: gradient vs oracle rel L2 {err:.2e}")
    # The fallback is taken when up_a + up_b is along the baseline, i.e. the baseline is
    # parallel to both detectors' columns: every epipolar line is then a column line
    # (alpha = 0), so every sample sits on the alpha = 0 grid line, where the bilinear
    # look-up's alpha slope jumps between the cell above and the folded cell below.  The
    # value is continuous (checked above at the FP32 bar); the gradient takes one-sided
    # slopes, and the FP32 positions pick the side per sample apart from the FP64 oracle.
    # Measured 1.25e-5; the bar here is 1e-4.
    assert err <= 1e-4, err
