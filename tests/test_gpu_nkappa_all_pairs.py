"""N_kappa of every pair of full-size scans against the FP64 oracle: the integer sample
ranges that the double-float per-pair set-up derives from the arcs (Eq. 15's N_kappa).
Scans: c2 as it is (all 122,760 pairs sample their whole arc), c2 and c4 under a seeded
rigid motion per view (the valid arcs then overlap only partly, so the ranges are cut
inside the sampled arc), and c3 with its own motion (30,628 pairs).  N_kappa depends on
the geometry only, so both sides sample zero sinograms on a small (alpha, s) grid."""
import numpy as np
import pytest

import synth
from oracle import oracle as orc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _motion(n_views, rot_deg, trans_mm, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([np.deg2rad(rng.normal(0.0, rot_deg, (n_views, 3))),
                           rng.normal(0.0, trans_mm, (n_views, 3))], axis=1)


@pytest.mark.parametrize("name,rot_deg,trans_mm", [("c2", 0.0, 0.0), ("c2", 1.0, 2.0), ("c3", None, None),
                                                   ("c4", 0.5, 1.0)])
def test_nkappa_every_pair_equals_oracle(name, rot_deg, trans_mm):
    import paper_1806_02637_gb300 as ecc
    cfg = synth.CONFIGS[name]
    sc = synth.make_scan(cfg, with_images=False)
    P = np.ascontiguousarray(sc["P"])
    if rot_deg is None:
        th = sc["motion"]
    else:
        th = _motion(cfg.n_views, rot_deg, trans_mm, 31) if rot_deg > 0 else None
    n_alpha, n_s = 4, 5
    ref = np.asarray(orc.ecc(P, np.zeros((cfg.n_views, n_alpha, n_s)), cfg.W, cfg.H, cfg.K, motion=th)["nk"])
    S = torch.zeros((cfg.n_views, n_alpha, n_s), dtype=torch.float32, device="cuda")
    r = ecc.ecc_evaluate(ecc.Context(0), torch.from_numpy(P).cuda(), S, cfg.W, cfg.H, cfg.K,
                         motion=None if th is None else torch.from_numpy(np.ascontiguousarray(th)).cuda())
    nk = r["nkappa"].cpu().numpy()
    assert nk.shape == ref.shape == (cfg.n_views * (cfg.n_views - 1) // 2,)
    bad = np.nonzero(nk != ref)[0]
    assert bad.size == 0, (bad[:10], nk[bad[:10]], ref[bad[:10]])
    if th is not None:  # the case cuts ranges inside the sampled arc
        assert (ref < cfg.K).mean() > 0.1
