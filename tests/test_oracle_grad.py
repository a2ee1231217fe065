"""Pins of the oracle gradient (complex-step differentiation of the total, Eq. 17,
with respect to per-view rigid motion) against central finite differences of the
forward oracle and against the null space of global rigid motion."""
import functools

import numpy as np

import synth
from oracle import oracle as orc
from tests import helpers as H

K = 96


@functools.lru_cache(maxsize=None)
def _scan():
    """Eight views of the 248-view motion workload, reduced sinogram grid."""
    cfg = synth.CONFIGS["c3"]
    sc = synth.make_scan(cfg, views=np.arange(0, 248, 31))
    S = orc.radon_derivative(sc["P"], sc["images"], 192, 256)
    return cfg, sc, S


def test_grad_vs_central_differences():
    cfg, sc, S = _scan()
    nv = len(sc["P"])
    th = sc["motion"]
    c = 50.0
    g = orc.ecc_grad(sc["P"], S, cfg.W, cfg.H, K, cauchy_c=c, motion=th)
    arcs = g["arcs"]
    rng = np.random.default_rng(32)
    picks = rng.choice(nv * 6, size=32, replace=False)
    # h = 1e-4 rad about the world origin moves lines by about 0.1 px, across the kinks
    # of the piecewise-bilinear look-up, so that bar is loose; the differences converge
    # to the complex-step values as h shrinks.
    for h, tol in ((1e-4, 0.35), (1e-6, 3e-3), (1e-7, 5e-4)):
        fd = []
        for q in picks:
            tp, tm = th.copy(), th.copy()
            tp.flat[q] += h
            tm.flat[q] -= h
            fp = orc.ecc(sc["P"], S, cfg.W, cfg.H, K, cauchy_c=c, motion=tp, arcs=arcs)["total"]
            fm = orc.ecc(sc["P"], S, cfg.W, cfg.H, K, cauchy_c=c, motion=tm, arcs=arcs)["total"]
            fd.append((fp - fm) / (2 * h))
        fd = np.array(fd)
        an = g["grad"].flat[picks]
        # piecewise-bilinear look-ups: central differences are exact only between kinks
        assert np.linalg.norm(fd - an) <= tol * np.linalg.norm(an), (h, np.linalg.norm(fd - an) / np.linalg.norm(an))
    # the forward part of the gradient call is the plain forward
    f = orc.ecc(sc["P"], S, cfg.W, cfg.H, K, cauchy_c=c, motion=th, arcs=arcs)
    assert np.isclose(g["total"], f["total"], rtol=1e-13)


def test_grad_global_rigid_null_space():
    """At theta = 0 a global rigid motion is the sum of the per-view motions; the
    total is invariant under it, so each column of the gradient sums to zero."""
    cfg, sc, S = _scan()
    rng = np.random.default_rng(4)
    Sn = S + rng.normal(0, 0.05 * np.abs(S).max(), S.shape)   # inconsistent data: nonzero gradient
    g = orc.ecc_grad(sc["P"], Sn, cfg.W, cfg.H, K)
    col = g["grad"].sum(axis=0)
    assert np.all(np.abs(col) <= 1e-7 * np.abs(g["grad"]).max(axis=0)), col / np.abs(g["grad"]).max(axis=0)
    assert np.abs(g["grad"]).max() > 0


# ------------------------------------------------ gradient w.r.t. the entries of P
# (geometric calibration by the consistency, Introduction): the view uses P T(theta)

def test_grad_P_vs_central_differences():
    cfg, sc, S = _scan()
    nv = len(sc["P"])
    th = sc["motion"]
    c = 50.0
    g = orc.ecc_grad_P(sc["P"], S, cfg.W, cfg.H, K, cauchy_c=c, motion=th)
    arcs = g["arcs"]
    rng = np.random.default_rng(33)
    picks = rng.choice(nv * 12, size=32, replace=False)
    for eps, tol in ((1e-6, 0.35), (1e-8, 3e-3), (1e-9, 5e-4)):
        steps = eps * H.p_entry_scale(sc["P"])
        fd, an = [], []
        for q in picks:
            h = steps.flat[q]
            Pp, Pm = sc["P"].reshape(nv, 12).copy(), sc["P"].reshape(nv, 12).copy()
            Pp.flat[q] += h
            Pm.flat[q] -= h
            fp = orc.ecc(Pp, S, cfg.W, cfg.H, K, cauchy_c=c, motion=th, arcs=arcs)["total"]
            fm = orc.ecc(Pm, S, cfg.W, cfg.H, K, cauchy_c=c, motion=th, arcs=arcs)["total"]
            fd.append((fp - fm) / (2 * h) * h)      # compared in units of the step
            an.append(g["grad"].flat[q] * h)
        fd, an = np.array(fd), np.array(an)
        assert np.linalg.norm(fd - an) <= tol * np.linalg.norm(an), (eps, np.linalg.norm(fd - an) / np.linalg.norm(an))
    f = orc.ecc(sc["P"], S, cfg.W, cfg.H, K, cauchy_c=c, motion=th, arcs=arcs)
    assert np.isclose(g["total"], f["total"], rtol=1e-13)


def test_grad_P_scale_invariance():
    """The total does not change under P_lambda -> s P_lambda (s > 0) for one view, so
    by Euler's theorem on homogeneous functions sum_ij P_ij dtotal/dP_ij = 0 per view."""
    cfg, sc, S = _scan()
    g = orc.ecc_grad_P(sc["P"], S, cfg.W, cfg.H, K, cauchy_c=20.0, motion=sc["motion"])["grad"]
    Pv = sc["P"].reshape(-1, 12)
    euler = (Pv * g).sum(axis=1)
    mag = np.abs(Pv * g).sum(axis=1)
    assert np.all(np.abs(euler) <= 1e-8 * mag), euler / mag
    assert np.all(mag > 0)


def test_grad_P_chain_rule_and_rigid_null_space():
    """(i) The gradient with respect to the unmoved P equals the one with respect to
    the moved P' = P T(theta) times T(theta)^T.  (ii) At theta = 0 the motion
    gradient is the P gradient contracted with d(P T(theta))/d theta_k, and the sum
    over views of that contraction vanishes for each rigid generator."""
    cfg, sc, S = _scan()
    nv = len(sc["P"])
    th = sc["motion"]
    Pv = sc["P"].reshape(nv, 12)
    g = orc.ecc_grad_P(Pv, S, cfg.W, cfg.H, K, motion=th)
    Pm = np.stack([orc.apply_motion(Pv[i], th[i]).reshape(12) for i in range(nv)])
    gm = orc.ecc_grad_P(Pm, S, cfg.W, cfg.H, K, arcs=g["arcs"])
    for i in range(nv):
        T = np.eye(4)
        T[:3, :] = orc.apply_motion(np.hstack([np.eye(3), np.zeros((3, 1))]).reshape(12), th[i]).reshape(3, 4)
        np.testing.assert_allclose(g["grad"][i].reshape(3, 4), gm["grad"][i].reshape(3, 4) @ T.T,
                                   rtol=1e-7, atol=1e-9 * np.abs(g["grad"][i]).max())
    # (ii) at theta = 0, with an inconsistent sinogram so that the gradient is not 0
    rng = np.random.default_rng(4)
    Sn = S + rng.normal(0, 0.05 * np.abs(S).max(), S.shape)
    gP = orc.ecc_grad_P(Pv, Sn, cfg.W, cfg.H, K)["grad"]
    gt = orc.ecc_grad(Pv, Sn, cfg.W, cfg.H, K)["grad"]
    # d(P T(theta))/d theta_k at theta = 0 is P G_k with the generators of R = Rz Ry Rx
    # (infinitesimal rotations about x, y, z) and of the translation
    gens = np.zeros((6, 4, 4))
    gens[0, 2, 1], gens[0, 1, 2] = 1.0, -1.0
    gens[1, 0, 2], gens[1, 2, 0] = 1.0, -1.0
    gens[2, 1, 0], gens[2, 0, 1] = 1.0, -1.0
    for k in range(3):
        gens[3 + k, k, 3] = 1.0
    for k in range(6):
        dP = np.stack([(Pv[i].reshape(3, 4) @ gens[k]).reshape(12) for i in range(nv)])
        contr = (gP * dP).sum(axis=1)
        np.testing.assert_allclose(contr, gt[:, k], rtol=1e-6, atol=1e-8 * np.abs(gt[:, k]).max())
        assert abs(contr.sum()) <= 1e-7 * np.abs(contr).max()
