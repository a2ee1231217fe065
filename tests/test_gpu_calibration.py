"""Geometric calibration by the consistency (the Introduction names calibration as a
use of the epipolar consistency): the gradient of the total (Eq. 17) with respect to
the 12 entries of each view's projection matrix, through the C ABI.

* parity with the oracle's complex-step gradient, compared in units of relative
  change of each entry;
* per-view scale invariance (Euler's identity) and the tie to the motion gradient,
  whose per-pair chain is separate code: contracted with the rigid generators, the
  P gradient is the motion gradient;
* central differences of the library's frozen forward;
* a refinement loop: detector row shifts of every view are removed by gradient
  steps on the entries of P."""
import functools

import numpy as np
import pytest

import synth
from oracle import oracle as orc
from tests import helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# the FP32 bar, as for the motion gradient: relative L2 error of the whole (scaled)
# gradient, and every component within TOL_GRAD of its norm.  Measured (GB300): 1.0e-7
# (c = 0) and 1.9e-7 (Cauchy c = median d) on the 20-view subset.
TOL_GRAD = 1e-5
VIEWS = tuple(range(0, 248, 13))   # 20 views of the 248-view motion workload


@functools.lru_cache(maxsize=None)
def _ctx():
    import paper_1806_02637_gb300 as ecc
    return ecc.Context(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _cudaP(P):
    return _cuda(np.asarray(P, dtype=np.float64).reshape(-1, 3, 4))


@functools.lru_cache(maxsize=None)
def _case():
    cfg = synth.CONFIGS["c3"]
    sc = H.scan("c3", VIEWS)
    S = H.oracle_sino("c3", VIEWS)
    return cfg, sc, S


def _gpu_grad_P(P, S32, W, Hh, K, c=0.0, motion=None, pairs=None):
    import paper_1806_02637_gb300 as ecc
    r = ecc.ecc_evaluate_grad_projection(_ctx(), _cudaP(P), _cuda(S32), W, Hh, K, cauchy_c=c,
                                         motion=None if motion is None else _cuda(motion),
                                         pairs=None if pairs is None else _cuda(np.asarray(pairs, np.int32)))
    torch.cuda.synchronize()
    return float(r["total"].cpu()[0]), r["grad_P"].cpu().numpy()


# rigid generators: d(P T(theta))/d theta_k at theta = 0 is P G_k (R = Rz Ry Rx)
GENS = np.zeros((6, 4, 4))
GENS[0, 2, 1], GENS[0, 1, 2] = 1.0, -1.0
GENS[1, 0, 2], GENS[1, 2, 0] = 1.0, -1.0
GENS[2, 1, 0], GENS[2, 0, 1] = 1.0, -1.0
for _k in range(3):
    GENS[3 + _k, _k, 3] = 1.0


@pytest.mark.parametrize("c", [0.0, "median"])
def test_grad_P_matches_oracle(c):
    cfg, sc, S = _case()
    S32 = S.astype(np.float32)
    th = sc["motion"]
    if c == "median":
        c = float(np.median(orc.ecc(sc["P"], S32.astype(np.float64), cfg.W, cfg.H, cfg.K, motion=th)["d"]))
    total, g = _gpu_grad_P(sc["P"], S32, cfg.W, cfg.H, cfg.K, c, th)
    ref = orc.ecc_grad_P(sc["P"], S32.astype(np.float64), cfg.W, cfg.H, cfg.K, cauchy_c=c, motion=th)
    s = H.p_entry_scale(sc["P"])
    gs, rs = g * s, ref["grad"] * s
    err = np.linalg.norm(gs - rs) / np.linalg.norm(rs)
    comp = np.abs(gs - rs).max() / np.linalg.norm(rs)
    print(f"calibration gradient vs oracle, c = {c}: rel L2 {err:.2e}, max component / norm {comp:.2e}")
    assert err <= TOL_GRAD and comp <= TOL_GRAD, (err, comp)
    assert abs(total - ref["total"]) <= H.TOL_F32 * ref["total"]


def test_grad_P_explicit_pairs():
    cfg, sc, S = _case()
    S32 = S.astype(np.float32)
    n = len(VIEWS)
    rng = np.random.default_rng(19)
    pairs = np.array([(a, b) for a in range(n) for b in range(n) if a != b])[rng.choice(n * (n - 1), 120, False)]
    _, g = _gpu_grad_P(sc["P"], S32, cfg.W, cfg.H, cfg.K, pairs=pairs)
    ref = orc.ecc_grad_P(sc["P"], S32.astype(np.float64), cfg.W, cfg.H, cfg.K, pairs=pairs)
    s = H.p_entry_scale(sc["P"])
    err = np.linalg.norm((g - ref["grad"]) * s) / np.linalg.norm(ref["grad"] * s)
    comp = np.abs((g - ref["grad"]) * s).max() / np.linalg.norm(ref["grad"] * s)
    print(f"calibration gradient vs oracle, explicit pairs: rel L2 {err:.2e}, max component / norm {comp:.2e}")
    assert err <= TOL_GRAD and comp <= TOL_GRAD, (err, comp)


def test_grad_P_euler_identity_and_motion_gradient():
    """On an inconsistent sinogram (nonzero gradient), at theta = 0: sum_ij P_ij g_ij
    = 0 per view (the total ignores the scale of each P), and the P gradient
    contracted with P G_k equals the motion gradient of ecc_evaluate_grad."""
    import paper_1806_02637_gb300 as ecc
    cfg, sc, S = _case()
    rng = np.random.default_rng(4)
    Sn = (S + rng.normal(0, 0.05 * np.abs(S).max(), S.shape)).astype(np.float32)
    n = len(VIEWS)
    Pv = sc["P"].reshape(n, 12)
    _, g = _gpu_grad_P(Pv, Sn, cfg.W, cfg.H, cfg.K)
    euler = (Pv * g).sum(axis=1)
    assert np.all(np.abs(euler) <= 1e-9 * np.abs(Pv * g).sum(axis=1)), euler
    r = ecc.ecc_evaluate_grad(_ctx(), _cudaP(Pv), _cuda(Sn), cfg.W, cfg.H, cfg.K)
    gt = r["grad"].cpu().numpy()
    for k in range(6):
        dP = np.stack([(Pv[i].reshape(3, 4) @ GENS[k]).reshape(12) for i in range(n)])
        np.testing.assert_allclose((g * dP).sum(axis=1), gt[:, k], rtol=1e-9, atol=1e-9 * np.abs(gt[:, k]).max())


def test_grad_P_vs_central_differences_of_frozen_forward():
    """Central differences of ecc_evaluate_frozen in P, steps of 1e-4 of each entry's
    scale (lines move by ~0.05 px, across the kinks of the bilinear look-up)."""
    import paper_1806_02637_gb300 as ecc
    cfg, sc, S = _case()
    S32 = _cuda(S.astype(np.float32))
    th = _cuda(sc["motion"])
    n = len(VIEWS)
    Pv = sc["P"].reshape(n, 12)
    r = ecc.ecc_evaluate_grad_projection(_ctx(), _cudaP(Pv), S32, cfg.W, cfg.H, cfg.K, motion=th)
    g = r["grad_P"].cpu().numpy()
    steps = 1e-4 * H.p_entry_scale(Pv)
    picks = np.random.default_rng(34).choice(Pv.size, 32, replace=False)
    fd, an = [], []
    for q in picks:
        vals = []
        for sgn in (1, -1):
            Pq = Pv.copy()
            Pq.flat[q] += sgn * steps.flat[q]
            rr = ecc.ecc_evaluate_frozen(_ctx(), _cudaP(Pq), S32, cfg.W, cfg.H, cfg.K, motion=th)
            torch.cuda.synchronize()
            vals.append(float(rr["total"].cpu()[0]))
        fd.append((vals[0] - vals[1]) / 2.0)
        an.append(g.flat[q] * steps.flat[q])
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) <= 0.35 * np.linalg.norm(an), np.linalg.norm(fd - an) / np.linalg.norm(an)
    assert fd @ an > 0


CAL = synth.ScanConfig("cal", n_views=40, arc_deg=200.0, full_scan=False, W=128, H=96, pixel_mm=2.0,
                       phantom="ellipsoids", n_prim=6, size_range=(10.0, 30.0), value_range=(0.1, 1.0),
                       n_alpha=128, n_s=161, K=128, seed=31)


def test_calibration_refinement_removes_detector_shifts():
    """Every view's detector is shifted by N(0, 1.5 px) rows; sinograms are computed
    with the shifted (wrong) matrices, as a scan with that calibration error would
    be.  Gradient steps on the entries of P (scaled per entry) lower the total to
    near the correctly calibrated one and reduce the reprojection error of points
    in the field of view (without its mean over views: a shift common to all views
    is a global motion, which the consistency cannot see)."""
    import paper_1806_02637_gb300 as ecc
    sc = synth.make_scan(CAL)
    n = CAL.n_views
    P0 = sc["P"].reshape(n, 3, 4)
    dv = np.random.default_rng(7).normal(0.0, 1.5, n)
    Pp = np.stack([np.array([[1, 0, 0], [0, 1, dv[i]], [0, 0, 1.0]]) @ P0[i] for i in range(n)]).reshape(n, 12)
    ctx = ecc.Context(0)
    S, _ = ecc.ecc_precompute_radon_derivative(ctx, _cudaP(Pp), _cuda(sc["images"]), CAL.n_alpha, CAL.n_s)
    ideal = float(ecc.ecc_evaluate(ctx, _cudaP(P0), S, CAL.W, CAL.H, CAL.K)["total"].cpu()[0])
    s2 = H.p_entry_scale(Pp) ** 2
    P = Pp.copy()
    totals = []
    eta = None
    for it in range(31):
        r = ecc.ecc_evaluate_grad_projection(ctx, _cudaP(P), S, CAL.W, CAL.H, CAL.K)
        totals.append(float(r["total"].cpu()[0]))
        g = r["grad_P"].cpu().numpy()
        if eta is None:   # the first step changes the most-affected entry by 1e-3 of its scale
            eta = 1e-3 / np.abs(np.sqrt(s2) * g).max()
        P = P - eta * s2 * g
    ctx.close()
    assert totals[-1] - ideal < 0.05 * (totals[0] - ideal), (totals[0], totals[-1], ideal)

    X = np.random.default_rng(1).uniform(-40.0, 40.0, (64, 3))
    Xh = np.hstack([X, np.ones((64, 1))])

    def reproj_rms(Pv):
        def proj(Q):
            x = np.einsum("vij,pj->vpi", Q.reshape(-1, 3, 4), Xh)
            return x[..., :2] / x[..., 2:]
        d = proj(Pv) - proj(P0)
        d = d - d.mean(axis=0, keepdims=True)
        return np.sqrt((d ** 2).sum(-1).mean())

    e0, e1 = reproj_rms(Pp), reproj_rms(P)
    assert e1 < 0.4 * e0, (e0, e1)
