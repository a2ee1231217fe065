"""One small, repeatable launch sequence per kernel family, for profilers.

    python profile_case.py --case radon  [--views 32]
    python profile_case.py --case pairs  [--views 128]
    python profile_case.py --case grad   [--views 128]

Each case builds a seeded subset of the 496-view short scan (620 x 480 detector,
768 x 768 dRadon/ds grid, 512 kappa), runs the call three times untimed and three
times with the library's per-kernel event timing, and prints those timings.  Under
a profiler, skip the first two launches of the kernel of interest (``-s 2``) to
capture a warm one.  The inputs stay well below a few GB of device memory.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["radon", "pairs", "grad"], required=True)
    ap.add_argument("--views", type=int, default=0, help="views of the short scan (default 32 / 128)")
    a = ap.parse_args(argv)
    import torch

    import synth
    import paper_1806_02637_gb300 as ecc

    cfg = synth.CONFIGS["c2"]
    if a.case == "radon":
        n = a.views or 32
        views = np.arange(0, cfg.n_views, 15)[:n]
    else:  # pairs, grad
        n = a.views or 128
        views = np.arange(0, cfg.n_views, max(1, cfg.n_views // n))[:n]
    sc = synth.make_scan(cfg, views=views)
    ctx = ecc.Context(0)
    P = torch.from_numpy(sc["P"]).cuda()
    im = torch.from_numpy(sc["images"]).cuda()

    # the gradient case: seeded rigid motion, rotations N(0, 1 deg), translations N(0, 2 mm)
    rng = np.random.default_rng(2024)
    motion = torch.from_numpy(np.concatenate([rng.normal(0.0, np.deg2rad(1.0), (len(views), 3)),
                                              rng.normal(0.0, 2.0, (len(views), 3))], axis=1)).cuda()

    def run():
        if a.case == "radon":
            return ecc.ecc_precompute_radon_derivative(ctx, P, im, cfg.n_alpha, cfg.n_s)
        if a.case == "grad":
            return ecc.ecc_evaluate_grad(ctx, P, S, cfg.W, cfg.H, cfg.K, motion=motion)
        return ecc.ecc_evaluate(ctx, P, S, cfg.W, cfg.H, cfg.K)

    S, _ = ecc.ecc_precompute_radon_derivative(ctx, P, im, cfg.n_alpha, cfg.n_s)
    if a.case in ("pairs", "grad"):
        del im
    torch.cuda.synchronize()
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    ecc.ecc_profile_enable(ctx, True)
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    print({k: (c, round(ms / max(c, 1), 4)) for k, (c, ms) in ecc.ecc_profile_read(ctx).items()})
    return 0


if __name__ == "__main__":
    sys.exit(main())
