"""Failure cases of the host and device paths through the C ABI: non-finite and
rank-deficient projection matrices, non-finite projection images.  Each is reported
(an error code, or a device status bit with the affected pairs left out as
N_kappa = 0, d = e = 0), the remaining pairs keep their values against the FP64
oracle, and the context stays usable afterwards.  Nothing here faults the GPU: the
failures are made in the inputs on the host."""
import functools
import time

import numpy as np
import pytest

import synth
from oracle import oracle as orc
from tests import helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CFG = synth.ScanConfig("fail", n_views=6, arc_deg=150.0, full_scan=False, W=96, H=80, pixel_mm=3.0,
                       phantom="blobs", n_prim=3, size_range=(10.0, 20.0), value_range=(0.01, 0.02),
                       n_alpha=96, n_s=121, K=64, seed=77)
BAD = 2   # the view that gets the bad input
DEGENERATE_VIEW, DEGENERATE_PAIR, NONFINITE_PAIR = 1, 2, 4


@functools.lru_cache(maxsize=None)
def _ctx():
    import paper_1806_02637_gb300 as ecc
    return ecc.Context(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@functools.lru_cache(maxsize=None)
def _scan():
    sc = synth.make_scan(CFG)
    return sc, orc.radon_derivative(sc["P"], sc["images"], CFG.n_alpha, CFG.n_s)


def _good_pairs():
    pairs = synth.upper_pairs(CFG.n_views)
    keep = (pairs[:, 0] != BAD) & (pairs[:, 1] != BAD)
    return pairs, keep


def _check_rest(r, P_ok, S_ok, motion=None):
    """Pairs without the bad view against the oracle; pairs with it dropped."""
    pairs, keep = _good_pairs()
    pp = r["per_pair"].cpu().numpy()
    nk = r["nkappa"].cpu().numpy()
    assert np.all(nk[~keep] == 0) and np.all(pp[~keep] == 0.0)
    ref = orc.ecc(P_ok, S_ok, CFG.W, CFG.H, CFG.K, motion=motion, pairs=pairs[keep])
    assert np.array_equal(nk[keep], ref["nk"])
    E = H.energies(P_ok, S_ok, CFG.W, CFG.H, CFG.K, pairs[keep], motion)
    assert H.pair_rel_err(pp[keep, 0], ref["d"], E).max() <= H.TOL_F32
    total = float(r["total"].cpu()[0])
    assert np.isfinite(total) and abs(total - ref["total"]) <= H.TOL_F32 * ref["total"]


def _still_usable():
    import paper_1806_02637_gb300 as ecc
    sc, S = _scan()
    r = ecc.ecc_evaluate(_ctx(), _cuda(sc["P"]), _cuda(S.astype(np.float32)), CFG.W, CFG.H, CFG.K)
    torch.cuda.synchronize()
    ref = orc.ecc(sc["P"], S.astype(np.float32).astype(np.float64), CFG.W, CFG.H, CFG.K)
    assert abs(float(r["total"].cpu()[0]) - ref["total"]) <= H.TOL_F32 * ref["total"]
    assert ecc.ecc_status(_ctx()) == 0


def _bad_P(kind):
    sc, _ = _scan()
    P = sc["P"].copy()
    if kind == "nan":
        P[BAD, 1, 2] = np.nan
    elif kind == "inf_t":
        P[BAD, 0, 3] = np.inf
    else:  # rank 2: the third row repeats the first
        P[BAD, 2] = P[BAD, 0]
    return P


@pytest.mark.parametrize("kind", ["nan", "inf_t", "rank2"])
def test_bad_projection_matrix_in_evaluate_and_gradient(kind):
    import paper_1806_02637_gb300 as ecc
    sc, S = _scan()
    P = _bad_P(kind)
    S32 = S.astype(np.float32)
    ecc.ecc_status(_ctx())
    r = ecc.ecc_evaluate(_ctx(), _cuda(P), _cuda(S32), CFG.W, CFG.H, CFG.K)
    torch.cuda.synchronize()
    assert ecc.ecc_status(_ctx()) & DEGENERATE_VIEW
    _check_rest(r, sc["P"], S32.astype(np.float64))
    g = ecc.ecc_evaluate_grad(_ctx(), _cuda(P), _cuda(S32), CFG.W, CFG.H, CFG.K)
    torch.cuda.synchronize()
    assert ecc.ecc_status(_ctx()) & DEGENERATE_VIEW
    grad = g["grad"].cpu().numpy()
    assert np.isfinite(grad).all() and np.all(grad[BAD] == 0.0)
    _still_usable()


def test_nonfinite_motion():
    import paper_1806_02637_gb300 as ecc
    sc, S = _scan()
    th = np.zeros((CFG.n_views, 6))
    th[BAD, 4] = np.nan
    ecc.ecc_status(_ctx())
    r = ecc.ecc_evaluate(_ctx(), _cuda(sc["P"]), _cuda(S.astype(np.float32)), CFG.W, CFG.H, CFG.K, motion=_cuda(th))
    torch.cuda.synchronize()
    assert ecc.ecc_status(_ctx()) & DEGENERATE_VIEW
    ok = th.copy()
    ok[BAD] = 0.0
    _check_rest(r, sc["P"], S.astype(np.float32).astype(np.float64), motion=ok)
    _still_usable()


def _nan_images():
    """A NaN detector row and column in the bad view: every line that meets its
    detector crosses one of them."""
    sc, _ = _scan()
    im = sc["images"].copy()
    im[BAD, 40, :] = np.nan
    im[BAD, :, 48] = np.nan
    return im


def test_nonfinite_images_in_precompute_evaluate_and_gradient():
    """NaN pixels reach the view's sinogram through the precompute; every pair with that
    view has a non-finite sum and is dropped with ECC_STATUS_NONFINITE_PAIR.  The other
    views take the oracle's sinograms, so that their pairs compare at the FP32 bar."""
    import paper_1806_02637_gb300 as ecc
    sc, S_or = _scan()
    P = _cuda(sc["P"])
    ecc.ecc_status(_ctx())
    S, _ = ecc.ecc_precompute_radon_derivative(_ctx(), P, _cuda(_nan_images()), CFG.n_alpha, CFG.n_s)
    torch.cuda.synchronize()
    good = [i for i in range(CFG.n_views) if i != BAD]
    assert not torch.isfinite(S[BAD]).all() and torch.isfinite(S[good]).all()
    S32 = S_or.astype(np.float32)
    S[good] = _cuda(S32[good])
    r = ecc.ecc_evaluate(_ctx(), P, S, CFG.W, CFG.H, CFG.K)
    torch.cuda.synchronize()
    assert ecc.ecc_status(_ctx()) & NONFINITE_PAIR
    _check_rest(r, sc["P"], S32.astype(np.float64))
    g = ecc.ecc_evaluate_grad(_ctx(), P, S, CFG.W, CFG.H, CFG.K)
    torch.cuda.synchronize()
    assert ecc.ecc_status(_ctx()) & NONFINITE_PAIR
    assert np.isfinite(g["grad"].cpu().numpy()).all()
    _still_usable()


def _serve(P, images, n_iters=3):
    import paper_1806_02637_gb300 as ecc
    ctx = ecc.Context(0)
    try:
        t = ecc.ecc_submit(ctx, P, images, CFG.W, CFG.H, CFG.n_alpha, CFG.n_s, CFG.K, n_iters=n_iters, step=1e-4)
        t0 = time.time()
        while True:
            r = ecc.ecc_poll(ctx, t)
            if r is not None:
                break
            assert time.time() - t0 < 60.0, "serving did not finish"
            time.sleep(0.002)
        # the context serves the next job normally
        sc, _ = _scan()
        t = ecc.ecc_submit(ctx, sc["P"], sc["images"], CFG.W, CFG.H, CFG.n_alpha, CFG.n_s, CFG.K, n_iters=1,
                           step=1e-4)
        while (r2 := ecc.ecc_poll(ctx, t)) is None:
            time.sleep(0.002)
        assert r2["flags"] == 0 and np.isfinite(r2["total_last"])
        return r
    finally:
        ctx.close()


def test_submit_rejects_nonfinite_geometry():
    import paper_1806_02637_gb300 as ecc
    sc, _ = _scan()
    ctx = ecc.Context(0)
    try:
        with pytest.raises(ecc.EccError, match="non-finite"):
            ecc.ecc_submit(ctx, _bad_P("nan"), sc["images"], CFG.W, CFG.H, CFG.n_alpha, CFG.n_s, CFG.K, n_iters=2,
                           step=1e-4)
        th = np.zeros((CFG.n_views, 6))
        th[BAD, 0] = np.inf
        with pytest.raises(ecc.EccError, match="non-finite"):
            ecc.ecc_submit(ctx, sc["P"], sc["images"], CFG.W, CFG.H, CFG.n_alpha, CFG.n_s, CFG.K, n_iters=2,
                           step=1e-4, motion0=th)
    finally:
        ctx.close()


def test_served_job_with_rank_deficient_view():
    r = _serve(_bad_P("rank2"), _scan()[0]["images"])
    assert r["flags"] & DEGENERATE_VIEW
    assert np.isfinite(r["total_first"]) and np.isfinite(r["total_last"])


def test_served_job_with_nonfinite_images():
    sc, S = _scan()
    r = _serve(sc["P"], _nan_images())
    assert r["flags"] & NONFINITE_PAIR
    assert np.isfinite(r["total_first"]) and np.isfinite(r["total_last"])
    np.testing.assert_allclose(r["motion"][BAD], 0.0)   # no gradient reached the view
