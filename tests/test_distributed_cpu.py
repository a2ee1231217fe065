"""The multi-GPU partition of the path (paper_1806_02637_gb300.distributed) on CPU:

* the view slices and the pair tiles cover every view and every pair a < b exactly
  once, for several scan sizes and rank counts, with balanced pair counts;
* two gloo ranks on 127.0.0.1 run the distributed composition with the FP64 oracle
  standing in for the kernels (test-only): each rank computes the sinograms of its view
  slice, all-gathers them, evaluates its pair tiles (the total and the motion gradient)
  and all-reduces in FP64.  The result equals the single-process oracle over all pairs.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1806_02637_gb300 import distributed as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("n_views,world", [(2, 1), (9, 2), (17, 3), (64, 4), (496, 8), (1240, 8)])
def test_partition_covers_every_pair_once(n_views, world):
    sl = D.view_slices(n_views, world)
    assert sl[0][0] == 0 and sl[-1][1] == n_views
    assert all(sl[k][1] == sl[k + 1][0] for k in range(world - 1))
    assert max(e - b for b, e in sl) - min(e - b for b, e in sl) <= 1
    got = np.concatenate([D.rank_pairs(n_views, world, r) for r in range(world)])
    assert np.all(got[:, 0] < got[:, 1])
    key = got[:, 0].astype(np.int64) * n_views + got[:, 1]
    assert len(np.unique(key)) == len(key) == n_views * (n_views - 1) // 2
    counts = [len(D.rank_pairs(n_views, world, r)) for r in range(world)]
    largest_tile = max(len(t) for t in D.pair_tiles(n_views, 4 * world))
    assert max(counts) - min(counts) <= largest_tile


_WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import numpy as np, torch, torch.distributed as dist
import synth
from oracle import oracle as orc
from paper_1806_02637_gb300 import distributed as D
cfg = synth.ScanConfig("dist", n_views=9, arc_deg=150.0, full_scan=False, W=64, H=48, pixel_mm=4.0,
                       phantom="blobs", n_prim=3, size_range=(10.0, 20.0), value_range=(0.01, 0.02),
                       n_alpha=64, n_s=81, K=48, seed=91, motion_rot_deg=0.5, motion_trans_mm=1.0)
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
sc = synth.make_scan(cfg)
b, e = D.view_slices(cfg.n_views, world)[rank]
local = torch.from_numpy(orc.radon_derivative(sc["P"][b:e], sc["images"][b:e], cfg.n_alpha, cfg.n_s))
sino = D.all_gather_views(local, cfg.n_views, world).numpy()
pairs = D.rank_pairs(cfg.n_views, world, rank, blocks_per_rank=2)
r = orc.ecc_grad(sc["P"], sino, cfg.W, cfg.H, cfg.K, motion=sc["motion"], pairs=pairs)
total, grad = D.all_reduce_sum_fp64(torch.tensor([r["total"]], dtype=torch.float64),
                                    torch.from_numpy(r["grad"]))
print(json.dumps({{"rank": rank, "pairs": int(len(pairs)), "total": float(total[0]),
                  "grad": grad.numpy().tolist()}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_equal_single_process():
    torch = pytest.importorskip("torch")
    import synth
    from oracle import oracle as orc
    port = _free_port()
    code = _WORKER.format(root=ROOT)
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    assert sum(o["pairs"] for o in outs) == 36 and all(o["pairs"] > 0 for o in outs)
    cfg = synth.ScanConfig("dist", n_views=9, arc_deg=150.0, full_scan=False, W=64, H=48, pixel_mm=4.0,
                           phantom="blobs", n_prim=3, size_range=(10.0, 20.0), value_range=(0.01, 0.02),
                           n_alpha=64, n_s=81, K=48, seed=91, motion_rot_deg=0.5, motion_trans_mm=1.0)
    sc = synth.make_scan(cfg)
    S = orc.radon_derivative(sc["P"], sc["images"], cfg.n_alpha, cfg.n_s)
    ref = orc.ecc_grad(sc["P"], S, cfg.W, cfg.H, cfg.K, motion=sc["motion"])
    for o in outs:   # every rank holds the reduced result
        assert np.isclose(o["total"], ref["total"], rtol=1e-12)
        np.testing.assert_allclose(np.array(o["grad"]), ref["grad"], rtol=1e-10, atol=1e-12 * np.abs(ref["grad"]).max())
