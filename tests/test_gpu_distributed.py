"""The multi-GPU partition through the library on one GPU (a box here has one GPU):

* the ranks' pair tiles evaluated one after the other on this GPU: the FP64 sum of the
  partial totals and motion gradients equals the evaluation of all pairs at once;
* sharded_consistency in a one-rank NCCL group (the collectives run, with one
  participant) equals the unsharded path bitwise for the sinograms and to FP64 summation
  order for the total and the gradient.
Ranks that wait on one another are never emulated on one GPU; the multi-rank
collectives are covered on CPU (gloo) in tests/test_distributed_cpu.py."""
import functools
import os
import socket

import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VIEWS = tuple(range(0, 248, 9))   # 28 views of the 248-view motion workload


@functools.lru_cache(maxsize=None)
def _ctx():
    import paper_1806_02637_gb300 as ecc
    return ecc.Context(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("world", [2, 3, 8])
def test_rank_partials_sum_to_the_whole(world):
    import paper_1806_02637_gb300 as ecc
    from paper_1806_02637_gb300 import distributed as D
    cfg = synth.CONFIGS["c3"]
    sc = H.scan("c3", VIEWS)
    P, th = _cuda(sc["P"]), _cuda(sc["motion"])
    S = _cuda(H.oracle_sino("c3", VIEWS).astype(np.float32))
    whole = ecc.ecc_evaluate_grad(_ctx(), P, S, cfg.W, cfg.H, cfg.K, motion=th)
    t_whole = float(whole["total"].cpu()[0])
    g_whole = whole["grad"].cpu().numpy()
    n = len(VIEWS)
    tot, grad = 0.0, np.zeros((n, 6))
    for r in range(world):
        pairs = _cuda(D.rank_pairs(n, world, r, blocks_per_rank=2))
        part = ecc.ecc_evaluate_grad(_ctx(), P, S, cfg.W, cfg.H, cfg.K, motion=th, pairs=pairs)
        tot += float(part["total"].cpu()[0])
        grad += part["grad"].cpu().numpy()
    assert abs(tot - t_whole) <= 1e-12 * abs(t_whole)
    np.testing.assert_allclose(grad, g_whole, rtol=0, atol=1e-9 * np.abs(g_whole).max())


def test_sharded_consistency_one_rank_nccl():
    import torch.distributed as dist
    import paper_1806_02637_gb300 as ecc
    from paper_1806_02637_gb300 import distributed as D
    cfg = synth.CONFIGS["c3"]
    sc = H.scan("c3", VIEWS)
    P, th, images = _cuda(sc["P"]), _cuda(sc["motion"]), _cuda(sc["images"])
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        t, g = D.sharded_consistency(_ctx(), P, images, cfg.W, cfg.H, cfg.n_alpha, cfg.n_s, cfg.K, 0, 1,
                                     motion=th, with_grad=True)
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    S, _ = ecc.ecc_precompute_radon_derivative(_ctx(), P, images, cfg.n_alpha, cfg.n_s)
    ref = ecc.ecc_evaluate_grad(_ctx(), P, S, cfg.W, cfg.H, cfg.K, motion=th)
    torch.cuda.synchronize()
    t_ref = float(ref["total"].cpu()[0])
    assert abs(float(t.cpu()[0]) - t_ref) <= 1e-12 * abs(t_ref)
    g_ref = ref["grad"].cpu().numpy()
    np.testing.assert_allclose(g.cpu().numpy(), g_ref, rtol=0, atol=1e-9 * np.abs(g_ref).max())
