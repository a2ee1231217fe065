"""ecc_evaluate_noalloc (static scratch, no device allocation) against the
context-based ecc_evaluate on the same device inputs: several calls in a row with
different shapes, each compared with ecc_evaluate's output, plus the limits of the
static scratch.  The file name sorts last so that the suite also runs it after
every other GPU test; it passes alone in a fresh process as well."""
import functools

import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@functools.lru_cache(maxsize=None)
def _ctx():
    import paper_1806_02637_gb300 as ecc
    return ecc.Context(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@functools.lru_cache(maxsize=None)
def _case(name):
    """Device inputs and the ecc_evaluate result of one workload."""
    import paper_1806_02637_gb300 as ecc
    if name == "c2-all":
        cfg, views, K, c, dtype = synth.CONFIGS["c2"], tuple(range(0, 496, 21)), 512, 0.0, torch.float32
    elif name == "c3-motion-pairs":
        cfg, views, K, c, dtype = synth.CONFIGS["c3"], tuple(range(0, 248, 15)), 256, 5.0, torch.float32
    elif name == "c4-k77-bf16":
        # n_kappa below 96: the 32-sample-tile forward kernel with a ragged last tile
        # (77 = 2 x 32 + 13), BF16 storage, opposed views (full-pi arcs)
        cfg, views, K, c, dtype = synth.CONFIGS["c4"], (0, 7, 310, 620, 627), 77, 0.0, torch.bfloat16
    else:  # "c1-f16"
        cfg, views, K, c, dtype = synth.CONFIGS["c1"], None, 256, 0.0, torch.float16
    sc = H.scan(cfg.name, views)
    P = _cuda(sc["P"])
    S, scales = ecc.ecc_precompute_radon_derivative(_ctx(), P, _cuda(sc["images"]), cfg.n_alpha, cfg.n_s,
                                                    dtype=dtype)
    motion = pairs = None
    if name == "c3-motion-pairs":
        motion = _cuda(sc["motion"])
        allp = synth.upper_pairs(len(sc["P"]))
        sel = np.random.default_rng(7).choice(len(allp), 60, replace=False)
        pairs = _cuda(np.asarray(allp[np.sort(sel)], dtype=np.int32))
    r = ecc.ecc_evaluate(_ctx(), P, S, cfg.W, cfg.H, K, cauchy_c=c, motion=motion, pairs=pairs, scales=scales)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in r.items()}
    n_pairs = ref["nkappa"].shape[0]
    return dict(cfg=cfg, K=K, c=c, P=P, S=S, scales=scales, motion=motion, pairs=pairs, n_pairs=n_pairs, ref=ref)


def _outputs(case):
    dev = case["S"].device
    return (torch.empty((1,), dtype=torch.float64, device=dev),
            torch.empty((case["n_pairs"], 2), dtype=torch.float64, device=dev),
            torch.empty((case["n_pairs"],), dtype=torch.int32, device=dev))


def _noalloc(case, out):
    import paper_1806_02637_gb300 as ecc
    total, pp, nk = out
    cfg = case["cfg"]
    ecc.ecc_evaluate_noalloc(case["P"], case["S"], cfg.W, cfg.H, case["K"], total, cauchy_c=case["c"],
                             motion=case["motion"], pairs=case["pairs"], scales=case["scales"], per_pair=pp,
                             nkappa=nk)


def _check(case, out):
    total, pp, nk = (t.cpu().numpy() for t in out)
    ref = case["ref"]
    assert np.array_equal(nk, ref["nkappa"])
    d_ref = ref["per_pair"][:, 0]
    den = np.maximum(np.abs(ref["per_pair"]), H.FLOOR * np.abs(d_ref).max() + 1e-300)
    err = np.abs(pp - ref["per_pair"]) / den
    assert err.max() <= H.TOL_F32, err.max()
    tot_ref = float(ref["total"][0])
    assert abs(float(total[0]) - tot_ref) <= H.TOL_F32 * max(abs(tot_ref), 1e-300), (float(total[0]), tot_ref)


def test_noalloc_matches_ecc_evaluate_on_calls_in_a_row():
    names = ["c2-all", "c3-motion-pairs", "c1-f16", "c4-k77-bf16"]
    cases = [_case(n) for n in names]
    outs = [_outputs(c) for c in cases]
    reps = [_outputs(c) for c in cases[:2]]
    torch.cuda.synchronize()
    # calls in a row on one stream with no host synchronisation between them (each
    # looks up the scratch address; the first may load the library's module)
    for case, out in zip(cases, outs):
        _noalloc(case, out)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    _noalloc(cases[0], reps[0])
    _noalloc(cases[1], reps[1])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 >= free0, (free0, free1)
    for case, out in zip(cases, outs):
        _check(case, out)
    for case, out in zip(cases[:2], reps):
        _check(case, out)


def test_noalloc_default_pairs_without_per_pair_outputs():
    import paper_1806_02637_gb300 as ecc
    case = _case("c2-all")
    cfg = case["cfg"]
    for _ in range(2):
        total = torch.empty((1,), dtype=torch.float64, device=case["S"].device)
        ecc.ecc_evaluate_noalloc(case["P"], case["S"], cfg.W, cfg.H, case["K"], total)
        torch.cuda.synchronize()
        tot_ref = float(case["ref"]["total"][0])
        assert abs(float(total.cpu()[0]) - tot_ref) <= H.TOL_F32 * abs(tot_ref)


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    import paper_1806_02637_gb300 as ecc
    dev = torch.device("cuda", 0)
    total = torch.zeros((1,), dtype=torch.float64, device=dev)
    # 513 views (limit 512)
    P = torch.zeros((513, 3, 4), dtype=torch.float64, device=dev)
    S = torch.zeros((513, 4, 2), dtype=torch.float32, device=dev)
    with pytest.raises(ecc.EccError, match="512"):
        ecc.ecc_evaluate_noalloc(P, S, 64, 64, 8, total)
    # 4097 alpha rows (limit 4096)
    P = torch.zeros((2, 3, 4), dtype=torch.float64, device=dev)
    S = torch.zeros((2, 4097, 2), dtype=torch.float32, device=dev)
    with pytest.raises(ecc.EccError, match="4096"):
        ecc.ecc_evaluate_noalloc(P, S, 64, 64, 8, total)
    # 276 pairs * ceil(65536 / 32) tiles > 131072
    case = _case("c2-all")
    with pytest.raises(ecc.EccError, match="131072"):
        ecc.ecc_evaluate_noalloc(case["P"], case["S"], case["cfg"].W, case["cfg"].H, 65536, total)
    torch.cuda.synchronize()
    assert float(total.cpu()[0]) == 0.0  # nothing was written
