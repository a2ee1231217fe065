"""Pins of the oracle gradient (complex-step differentiation of the total, Eq. 17,
with respect to per-view rigid motion) against central finite differences of the
forward oracle and against the null space of global rigid motion."""
import functools

import numpy as np

import synth
from oracle import oracle as orc

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
