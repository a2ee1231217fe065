"""Host-side logic of serving that needs no GPU: the device-memory footprint a job
is admitted with, and argument validation of a job."""
import numpy as np
import pytest

import synth
import paper_1806_02637_gb300 as ecc

CFG = synth.ScanConfig("srv", n_views=6, arc_deg=120.0, full_scan=False, W=64, H=48, pixel_mm=4.0,
                       phantom="blobs", n_prim=2, size_range=(8.0, 12.0), value_range=(0.01, 0.02),
                       n_alpha=64, n_s=81, K=64, seed=11)


def _fp(**kw):
    sc = synth.make_scan(CFG, with_images=False)
    n = kw.pop("n", CFG.n_views)
    P = sc["P"][:n]
    images = np.zeros((n, CFG.H, CFG.W), np.float32)
    args = dict(W=CFG.W, H=CFG.H, n_alpha=CFG.n_alpha, n_s=CFG.n_s, n_kappa=CFG.K, n_iters=5, step=1e-3)
    args.update(kw)
    return ecc.ecc_job_footprint(P, images, **args)


def r256(x):
    return (x + 255) // 256 * 256


def test_footprint_sections():
    n = CFG.n_views
    base = _fp()
    # sinogram storage: BF16 halves the FP32 section (no staging for BF16)
    sino32, sino16 = n * CFG.n_alpha * CFG.n_s * 4, n * CFG.n_alpha * CFG.n_s * 2
    assert base - _fp(dtype="bfloat16") == r256(sino32) - r256(sino16)
    # FP16 adds its FP32 staging of one precompute batch (here all views) to the transient part
    # (an empty section still takes one 256-byte slot)
    assert _fp(dtype="float16") - _fp(dtype="bfloat16") == r256(n * CFG.n_alpha * CFG.n_s * 4) - 256
    # totals: n_iters + 1 doubles
    assert _fp(n_iters=500) - base == r256(501 * 8) - r256(6 * 8)
    # tile directions: n_pairs x ceil(K / 32) x 16 bytes
    npairs = n * (n - 1) // 2
    assert _fp(n_kappa=96) - base == r256(npairs * 3 * 16) - r256(npairs * 2 * 16)
    # grows with the views
    assert _fp(n=5) < base


@pytest.mark.parametrize("bad", [dict(n=1), dict(n_kappa=0), dict(dtype=5), dict(n_iters=-1),
                                 dict(step=float("nan")), dict(n_alpha=2)])
def test_invalid_jobs_rejected(bad):
    with pytest.raises(ecc.EccError):
        _fp(**bad)
