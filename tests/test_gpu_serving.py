"""Serving (continuous batching of motion-compensation jobs) through the C ABI:

* every job's results are the same when it is served alone and in a mix of jobs of
  other sizes, storage types and iteration counts (bit for bit: per-job reductions
  have a fixed order), and the mix really shares rounds;
* the served iterations equal a host-driven loop over ecc_evaluate_grad with the
  steps theta <- theta - step * grad (to the rounding of separately compiled
  copies of the FP32 per-sample code);
* admission by device-memory budget queues jobs that do not fit yet and rejects a
  job that never fits;
* the served totals match the FP64 oracle at the first and the final motion."""
import functools
import time

import numpy as np
import pytest

import synth
from oracle import oracle as orc
from tests import helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _cfg(name, n, W, Hh, n_alpha, n_s, K, seed):
    return synth.ScanConfig(name, n_views=n, arc_deg=150.0, full_scan=False, W=W, H=Hh, pixel_mm=3.0,
                            phantom="blobs", n_prim=3, size_range=(10.0, 20.0), value_range=(0.01, 0.02),
                            n_alpha=n_alpha, n_s=n_s, K=K, seed=seed, motion_rot_deg=0.5, motion_trans_mm=1.0)


# (config, dtype, n_iters, step, cauchy_c, with initial motion)
JOBS = {
    "A": (_cfg("sA", 8, 96, 80, 96, 121, 64, 21), "float32", 24, 2e-4, 0.0, True),
    "B": (_cfg("sB", 12, 128, 96, 128, 161, 96, 22), "float16", 16, 1e-4, 0.0, False),
    "C": (_cfg("sC", 6, 80, 80, 80, 113, 40, 23), "bfloat16", 30, 3e-4, 0.0, True),
    "D": (_cfg("sD", 10, 96, 64, 96, 115, 128, 24), "float32", 20, 1e-4, 5.0, True),
}


@functools.lru_cache(maxsize=None)
def _scan(name):
    cfg = JOBS[name][0]
    return synth.make_scan(cfg)


def _submit(ctx, name):
    import paper_1806_02637_gb300 as ecc
    cfg, dtype, iters, step, c, mot = JOBS[name]
    sc = _scan(name)
    return ecc.ecc_submit(ctx, sc["P"], sc["images"], cfg.W, cfg.H, cfg.n_alpha, cfg.n_s, cfg.K, n_iters=iters,
                          step=step, dtype=dtype, cauchy_c=c, motion0=sc["motion"] if mot else None)


def _wait(ctx, tickets, timeout=120.0):
    import paper_1806_02637_gb300 as ecc
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for name, t in tickets.items():
            if name not in out:
                r = ecc.ecc_poll(ctx, t)
                if r is not None:
                    out[name] = r
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.002)
    return out


@functools.lru_cache(maxsize=None)
def _alone():
    import paper_1806_02637_gb300 as ecc
    ctx = ecc.Context(0)
    res = {}
    for name in JOBS:
        res.update(_wait(ctx, {name: _submit(ctx, name)}))
    st = ecc.ecc_serve_stats(ctx)
    ctx.close()
    return res, st


def test_alone_equals_mix():
    import paper_1806_02637_gb300 as ecc
    alone, st_alone = _alone()
    assert st_alone["max_batch"] == 1
    ctx = ecc.Context(0)
    tickets = {name: _submit(ctx, name) for name in JOBS}
    mix = _wait(ctx, tickets)
    st = ecc.ecc_serve_stats(ctx)
    ctx.close()
    assert st["max_batch"] >= 2, st  # jobs shared rounds
    for name in JOBS:
        a, m = alone[name], mix[name]
        assert m["status"] == 0 and m["iters"] == JOBS[name][2]
        assert np.array_equal(a["totals"], m["totals"]), name
        assert np.array_equal(a["motion"], m["motion"]), name
        assert m["line_pairs"] == a["line_pairs"] > 0
        assert m["latency_ms"] >= m["queue_ms"] >= 0.0


@pytest.mark.parametrize("name", ["A", "B"])
def test_served_equals_host_loop(name):
    import paper_1806_02637_gb300 as ecc
    alone, _ = _alone()
    cfg, dtype, iters, step, c, mot = JOBS[name]
    sc = _scan(name)
    ctx = ecc.Context(0)
    P = torch.from_numpy(sc["P"]).cuda()
    S, scales = ecc.ecc_precompute_radon_derivative(ctx, P, torch.from_numpy(sc["images"]).cuda(), cfg.n_alpha,
                                                    cfg.n_s, dtype=getattr(torch, dtype))
    theta = torch.from_numpy(sc["motion"] if mot else np.zeros((cfg.n_views, 6))).cuda()
    totals = []
    for it in range(iters + 1):
        r = ecc.ecc_evaluate_grad(ctx, P, S, cfg.W, cfg.H, cfg.K, cauchy_c=c, motion=theta, scales=scales)
        totals.append(float(r["total"].cpu()[0]))
        if it < iters:
            theta = theta - step * r["grad"]
    theta = theta.cpu().numpy()
    ctx.close()
    served = alone[name]
    # the serving kernel and the single-scan kernel are separately compiled copies of
    # the same per-pair code and may round FP32 operations differently (1e-7 of the
    # larger pair values): held to the FP32 path's bar, and motion to 1e-8 rad / mm
    np.testing.assert_allclose(served["totals"], totals, rtol=H.TOL_F32, atol=0)
    np.testing.assert_allclose(served["motion"], theta, rtol=1e-6, atol=1e-8)


def test_admission_budget_and_reject():
    """Budget of one job A plus 4 KB: a second copy of A cannot be admitted while the
    first holds its resident memory, so it queues until the first is done."""
    import paper_1806_02637_gb300 as ecc
    alone, _ = _alone()
    cfg, dtype, iters, step, c, mot = JOBS["A"]
    sc = _scan("A")
    fa = ecc.ecc_job_footprint(sc["P"], sc["images"], cfg.W, cfg.H, cfg.n_alpha, cfg.n_s, cfg.K, iters, step,
                               dtype, c, sc["motion"])
    ctx = ecc.Context(0, hbm_budget_bytes=fa + 4096)
    tickets = {"A1": _submit(ctx, "A"), "A2": _submit(ctx, "A")}
    out = _wait(ctx, tickets)
    st = ecc.ecc_serve_stats(ctx)
    assert st["max_batch"] == 1, st
    assert st["rounds"] == 2 * (iters + 1), st
    for name in tickets:
        assert np.array_equal(out[name]["totals"], alone["A"]["totals"])
        assert out[name]["footprint_bytes"] == fa
    # a job larger than the whole budget is refused at submission
    big = _cfg("sBig", 40, 128, 128, 128, 181, 64, 25)
    scg = synth.make_scan(big, with_images=False)
    imgs = np.zeros((big.n_views, big.H, big.W), np.float32)
    with pytest.raises(ecc.EccError, match=r"\(-5\)"):
        ecc.ecc_submit(ctx, scg["P"], imgs, big.W, big.H, big.n_alpha, big.n_s, big.K, n_iters=2)
    ctx.close()


def test_served_totals_match_oracle():
    """Job A (FP32 storage): the served total at theta_0 and at the final theta equals
    the FP64 oracle on the library's sinograms at those motions (per-pair bar of the
    FP32 path, summed)."""
    import paper_1806_02637_gb300 as ecc
    alone, _ = _alone()
    cfg, dtype, iters, step, c, mot = JOBS["A"]
    sc = _scan("A")
    ctx = ecc.Context(0)
    S, _ = ecc.ecc_precompute_radon_derivative(ctx, torch.from_numpy(sc["P"]).cuda(),
                                               torch.from_numpy(sc["images"]).cuda(), cfg.n_alpha, cfg.n_s)
    S = S.cpu().numpy().astype(np.float64)
    ctx.close()
    served = alone["A"]
    for theta, total in ((sc["motion"], served["totals"][0]), (served["motion"], served["totals"][-1])):
        ref = orc.ecc(sc["P"], S, cfg.W, cfg.H, cfg.K, motion=theta, cauchy_c=c)
        E = H.energies(sc["P"], S, cfg.W, cfg.H, cfg.K, ref["pairs"], theta)
        bound = H.TOL_F32 * np.maximum(ref["e"], H.FLOOR * E).sum()
        assert abs(total - ref["total"]) <= bound, (total, ref["total"], bound)


def test_destroy_with_jobs_in_flight():
    """Destroying the context while jobs are queued and running drops them and returns
    (the scheduler threads stop after the GPU work already issued); a new context
    serves normally afterwards.  Unknown tickets are refused."""
    import paper_1806_02637_gb300 as ecc
    cfg, dtype, iters, step, c, mot = JOBS["A"]
    sc = _scan("A")
    ctx = ecc.Context(0)
    for _ in range(6):
        ecc.ecc_submit(ctx, sc["P"], sc["images"], cfg.W, cfg.H, cfg.n_alpha, cfg.n_s, cfg.K, n_iters=500,
                       step=step)
    time.sleep(0.05)
    t0 = time.time()
    ctx.close()
    assert time.time() - t0 < 30.0
    alone, _ = _alone()
    ctx = ecc.Context(0)
    with pytest.raises(ecc.EccError, match=r"\(-1\)"):
        ecc.ecc_poll(ctx, 12345)
    out = _wait(ctx, {"A": _submit(ctx, "A")})
    assert np.array_equal(out["A"]["totals"], alone["A"]["totals"])
    ctx.close()
