"""Multi-GPU form of the consistency (one process per GPU, torch.distributed).

Eq. 17 sums independent pair terms, and each view's S (Eq. 1) depends on that view
alone, so the path splits in two exchange steps:

1. the views are split into contiguous slices, one per rank; each rank computes the
   dRadon/ds sinograms of its slice, and an all-gather gives every rank all of them
   (on one GB300 the 496-view scan's FP32 sinograms are 1.17 GB, the 1240-view
   scan's FP16 ones 2.8 GB: every rank can hold all of them);
2. the upper-triangular pair matrix is cut into view-block x view-block tiles and
   the tiles are dealt to the ranks, balanced by pair count; a rank evaluates its
   tiles' pairs (neighbouring views: their sinogram curves share L2), and one FP64
   all-reduce sums the partial totals and gradients.

The compute of each step is the library's (ecc_precompute_radon_derivative,
ecc_evaluate, ecc_evaluate_grad); this module holds only the partition and the
collectives.  With NCCL on GPUs the collectives move device tensors; the same
functions run over gloo with CPU tensors.
"""
from __future__ import annotations

import numpy as np


def view_slices(n_views: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [begin, end) view ranges, one per rank, sizes differing by at most 1."""
    if world < 1:
        raise ValueError("world must be >= 1")
    q, r = divmod(n_views, world)
    out, b = [], 0
    for k in range(world):
        e = b + q + (1 if k < r else 0)
        out.append((b, e))
        b = e
    return out


def pair_tiles(n_views: int, n_blocks: int) -> list[np.ndarray]:
    """The pairs a < b of n_views views in view-block x view-block tiles (block i <=
    block j), each tile's pairs in row-major order: int32 [n, 2] arrays, together
    every pair exactly once."""
    n_blocks = max(1, min(n_blocks, n_views))
    edges = np.linspace(0, n_views, n_blocks + 1).round().astype(int)
    tiles = []
    for i in range(n_blocks):
        for j in range(i, n_blocks):
            a = np.arange(edges[i], edges[i + 1])
            b = np.arange(edges[j], edges[j + 1])
            A, B = np.meshgrid(a, b, indexing="ij")
            keep = A < B
            t = np.stack([A[keep], B[keep]], axis=1).astype(np.int32)
            if len(t):
                tiles.append(t)
    return tiles


def rank_pairs(n_views: int, world: int, rank: int, blocks_per_rank: int = 4) -> np.ndarray:
    """The pairs rank `rank` of `world` evaluates: tiles of pair_tiles(n_views,
    blocks_per_rank * world) dealt largest first to the rank with the fewest pairs so
    far (ties: the lowest rank), so that the ranks' pair counts differ by at most one
    tile.  int32 [n, 2]; the ranks' lists together hold every pair exactly once."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    tiles = pair_tiles(n_views, blocks_per_rank * world)
    order = sorted(range(len(tiles)), key=lambda t: (-len(tiles[t]), t))
    load = [0] * world
    mine = []
    for t in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += len(tiles[t])
        if r == rank:
            mine.append(t)
    mine.sort()
    if not mine:
        return np.zeros((0, 2), dtype=np.int32)
    return np.concatenate([tiles[t] for t in mine]).astype(np.int32)


def all_gather_views(local, n_views: int, world: int, group=None):
    """All-gather of per-rank view slices (view_slices order) along dim 0: `local` holds
    this rank's slice; returns the [n_views, ...] tensor of all views.  Slices are
    padded to the largest one for the collective."""
    import torch
    import torch.distributed as dist
    sl = view_slices(n_views, world)
    m = max(e - b for b, e in sl)
    pad = local.new_zeros((m,) + tuple(local.shape[1:]))
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[k][: e - b] for k, (b, e) in enumerate(sl)], dim=0)


def all_reduce_sum_fp64(total, grad=None, group=None):
    """Sum of the partial totals (and gradients) of all ranks in FP64, in one
    all-reduce of (total, grad) packed together.  Returns (total, grad)."""
    import torch
    import torch.distributed as dist
    parts = [total.reshape(-1).to(torch.float64)]
    if grad is not None:
        parts.append(grad.reshape(-1).to(torch.float64))
    buf = torch.cat(parts)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    t = buf[: parts[0].numel()].reshape(total.shape)
    g = None if grad is None else buf[parts[0].numel():].reshape(grad.shape)
    return t, g


def sharded_consistency(ctx, P, images, W: int, H: int, n_alpha: int, n_s: int, n_kappa: int, rank: int,
                        world: int, cauchy_c: float = 0.0, motion=None, dtype=None, with_grad: bool = False,
                        group=None, blocks_per_rank: int = 4):
    """The whole path on `world` GPUs, this process being `rank`: the precompute of
    this rank's view slice, the all-gather of the sinograms, the evaluation (with the
    motion gradient if with_grad) of this rank's pair tiles, and the FP64 all-reduce.
    P [N,3,4] float64 and images [N,H,W] float32 on this rank's GPU (all views).
    Returns (total [1] float64, grad [N,6] float64 or None), equal on every rank.
    FP16 storage is not offered here: its per-view scales would need their own
    all-gather."""
    import torch
    from . import ecc_evaluate, ecc_evaluate_grad, ecc_precompute_radon_derivative
    dtype = dtype or torch.float32
    if dtype == torch.float16:
        raise ValueError("sharded_consistency takes FP32 or BF16 storage")
    n = P.shape[0]
    b, e = view_slices(n, world)[rank]
    local, _ = ecc_precompute_radon_derivative(ctx, P[b:e], images[b:e], n_alpha, n_s, dtype=dtype)
    sino = all_gather_views(local, n, world, group)
    pairs = torch.from_numpy(rank_pairs(n, world, rank, blocks_per_rank)).to(P.device)
    if with_grad:
        r = ecc_evaluate_grad(ctx, P, sino, W, H, n_kappa, cauchy_c=cauchy_c, motion=motion, pairs=pairs,
                              want_per_pair=False)
        return all_reduce_sum_fp64(r["total"], r["grad"], group)
    r = ecc_evaluate(ctx, P, sino, W, H, n_kappa, cauchy_c=cauchy_c, motion=motion, pairs=pairs,
                     want_per_pair=False)
    return all_reduce_sum_fp64(r["total"], None, group)
