"""The Akima spline motion model in serving (Optimization section), on the GPU:

* a served spline job equals a host-driven loop in which theta comes from the
  oracle's spline of the node values, the gradient from ecc_evaluate_grad and the
  node step from the oracle's chain rule (totals at the FP32 bar);
* the paper's setting: z translations only, an injected smooth motion of 9 spline
  nodes on a short scan; gradient steps on the nodes lower the total and remove most
  of the injected motion."""
import time

import numpy as np
import pytest

import synth
from oracle import motion as mo
from tests import helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CFG = synth.ScanConfig("mot", n_views=40, arc_deg=200.0, full_scan=False, W=128, H=96, pixel_mm=2.0,
                       phantom="ellipsoids", n_prim=6, size_range=(10.0, 30.0), value_range=(0.1, 1.0),
                       n_alpha=128, n_s=161, K=128, seed=31)


def _wait(ctx, t, timeout=120.0):
    import paper_1806_02637_gb300 as ecc
    t0 = time.time()
    while True:
        r = ecc.ecc_poll(ctx, t)
        if r is not None:
            return r
        assert time.time() - t0 < timeout
        time.sleep(0.002)


def _scan():
    return synth.make_scan(CFG)


def test_spline_job_equals_host_loop():
    import paper_1806_02637_gb300 as ecc
    sc = _scan()
    n, n_nodes, mask, iters = CFG.n_views, 7, 0b100110, 6
    base = np.random.default_rng(3).normal(0.0, 0.3, (n, 6)) * np.array([0.01, 0.01, 0.01, 1, 1, 1])
    ctx = ecc.Context(0)
    # step from the initial node gradient: the largest node moves by 1e-3 (mm or rad), a
    # well-conditioned descent (rotations and translations share one step size)
    P = torch.from_numpy(sc["P"]).cuda()
    S, _ = ecc.ecc_precompute_radon_derivative(ctx, P, torch.from_numpy(sc["images"]).cuda(), CFG.n_alpha, CFG.n_s)
    # start from generic node values: with all nodes equal Akima's weights are 0/0 and
    # the spline has kinks, where one-sided derivatives (the oracle's differences)
    # and the library's equal-weights derivative need not agree
    nodes0 = np.random.default_rng(5).normal(0.0, 1.0, (n_nodes, 6)) * np.array([0.005] * 3 + [0.5] * 3)
    th0 = mo.spline_motion(n, nodes0, base, mask)
    g0 = ecc.ecc_evaluate_grad(ctx, P, S, CFG.W, CFG.H, CFG.K, motion=torch.from_numpy(th0).cuda())["grad"]
    step = 1e-3 / np.abs(mo.node_gradient(n, nodes0, g0.cpu().numpy(), mask)).max()
    t = ecc.ecc_submit(ctx, sc["P"], sc["images"], CFG.W, CFG.H, CFG.n_alpha, CFG.n_s, CFG.K, n_iters=iters,
                       step=step, motion0=base, motion_model="akima", n_nodes=n_nodes, param_mask=mask,
                       nodes0=nodes0)
    served = _wait(ctx, t)
    nodes = nodes0.copy()
    totals = []
    for it in range(iters + 1):
        th = mo.spline_motion(n, nodes, base, mask)
        r = ecc.ecc_evaluate_grad(ctx, P, S, CFG.W, CFG.H, CFG.K, motion=torch.from_numpy(th).cuda())
        totals.append(float(r["total"].cpu()[0]))
        if it < iters:
            nodes = nodes - step * mo.node_gradient(n, nodes, r["grad"].cpu().numpy(), mask)
    ctx.close()
    np.testing.assert_allclose(served["totals"], totals, rtol=H.TOL_F32, atol=0)
    # node values: two FP32 gradient evaluations (separately compiled per-sample code,
    # ~1e-6 apart) and the oracle's difference Jacobian, over six steps
    np.testing.assert_allclose(served["nodes"], nodes, rtol=1e-4, atol=1e-7)
    # the served motion is the library's FP64 spline of its own nodes (Akima's weights
    # amplify the node differences above where slopes nearly agree, so the motion is
    # compared at the served nodes)
    np.testing.assert_allclose(served["motion"], mo.spline_motion(n, served["nodes"], base, mask), rtol=1e-9,
                               atol=1e-12)
    # parameters outside the mask stay at motion0
    assert np.array_equal(served["motion"][:, [0, 3, 4]], base[:, [0, 3, 4]])


def test_z_translation_recovery():
    """Injected z translation (9 Akima nodes, N(0, 2 mm)); estimate tz only."""
    import paper_1806_02637_gb300 as ecc
    sc = _scan()
    n, n_nodes = CFG.n_views, 9
    rng = np.random.default_rng(4)
    true_nodes = np.zeros((n_nodes, 6))
    true_nodes[:, 5] = rng.normal(0.0, 2.0, n_nodes)
    injected = mo.spline_motion(n, true_nodes, None, 0b100000)
    ctx = ecc.Context(0)
    # step: the first move of the largest node is 0.5 mm
    P = torch.from_numpy(sc["P"]).cuda()
    S, _ = ecc.ecc_precompute_radon_derivative(ctx, P, torch.from_numpy(sc["images"]).cuda(), CFG.n_alpha, CFG.n_s)
    g0 = ecc.ecc_evaluate_grad(ctx, P, S, CFG.W, CFG.H, CFG.K, motion=torch.from_numpy(injected).cuda())["grad"]
    gn = mo.node_gradient(n, np.zeros((n_nodes, 6)), g0.cpu().numpy(), 0b100000)
    step = 0.5 / np.abs(gn[:, 5]).max()
    t = ecc.ecc_submit(ctx, sc["P"], sc["images"], CFG.W, CFG.H, CFG.n_alpha, CFG.n_s, CFG.K, n_iters=40,
                       step=step, motion0=injected, motion_model="akima", n_nodes=n_nodes, param_mask=0b100000)
    r = _wait(ctx, t)
    ideal = float(ecc.ecc_evaluate(ctx, P, S, CFG.W, CFG.H, CFG.K)["total"].cpu()[0])  # true geometry
    ctx.close()
    tot = r["totals"]
    assert tot[-1] - ideal < 0.5 * (tot[0] - ideal), (tot[0], tot[-1], ideal)
    # a z shift common to all views is a global rigid motion: the consistency cannot
    # see it, so the recovered motion is compared without its mean
    def rms(z):
        return np.sqrt(np.mean((z - z.mean()) ** 2))
    rms0, rms1 = rms(injected[:, 5]), rms(r["motion"][:, 5])
    assert rms1 < 0.5 * rms0, (rms0, rms1)


def test_paper_setting_z_translation_17_nodes():
    """The paper's motion experiment in shape (Optimization section): z translations only, 17 Akima
    nodes, on the 496-view 200-degree short scan (620x480 detector).  An injected smooth z motion
    (17 nodes, N(0, 2 mm)) is estimated by the served gradient loop; the excess total over the
    correctly calibrated geometry and the mean-free z error both drop by more than half."""
    import paper_1806_02637_gb300 as ecc
    cfg = synth.CONFIGS["c2"]
    sc = synth.make_scan(cfg)
    n, n_nodes = cfg.n_views, 17
    rng = np.random.default_rng(17)
    true_nodes = np.zeros((n_nodes, 6))
    true_nodes[:, 5] = rng.normal(0.0, 2.0, n_nodes)
    injected = mo.spline_motion(n, true_nodes, None, 0b100000)
    ctx = ecc.Context(0)
    P = torch.from_numpy(sc["P"]).cuda()
    S, _ = ecc.ecc_precompute_radon_derivative(ctx, P, torch.from_numpy(sc["images"]).cuda(), cfg.n_alpha, cfg.n_s)
    g0 = ecc.ecc_evaluate_grad(ctx, P, S, cfg.W, cfg.H, cfg.K, motion=torch.from_numpy(injected).cuda())["grad"]
    gn = mo.node_gradient(n, np.zeros((n_nodes, 6)), g0.cpu().numpy(), 0b100000)
    step = 0.5 / np.abs(gn[:, 5]).max()      # the first move of the largest node is 0.5 mm
    t = ecc.ecc_submit(ctx, sc["P"], sc["images"], cfg.W, cfg.H, cfg.n_alpha, cfg.n_s, cfg.K, n_iters=40,
                       step=step, motion0=injected, motion_model="akima", n_nodes=n_nodes, param_mask=0b100000)
    r = _wait(ctx, t, timeout=300.0)
    ideal = float(ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K)["total"].cpu()[0])
    ctx.close()
    tot = r["totals"]
    assert tot[-1] - ideal < 0.5 * (tot[0] - ideal), (tot[0], tot[-1], ideal)

    def rms(z):
        return np.sqrt(np.mean((z - z.mean()) ** 2))
    rms0, rms1 = rms(injected[:, 5]), rms(r["motion"][:, 5])
    print(f"z motion: mean-free RMS {rms0:.3f} mm -> {rms1:.3f} mm; excess total {tot[0] - ideal:.4g} -> "
          f"{tot[-1] - ideal:.4g}; latency {r['latency_ms']:.0f} ms")
    assert rms1 < 0.5 * rms0, (rms0, rms1)
