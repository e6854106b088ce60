"""Several GPUs, one process each: the batch of moves split across ranks.

Moves are independent once the block model and the schedule are fixed, so a
batch partitions into contiguous slices, one per rank, with move indices kept
global.  Each rank evaluates its slice and selects its own top k; the only
exchange is an all-gather of the ranks' k (index, score) keys, after which
every rank selects the batch's top k from the gathered candidates with the
library's top-k kernel and applies the same best move to its replica of the
state, so all replicas stay identical.  (When every rank searches its own
independent batch, nothing is exchanged at all.)

The merge is exact: ranks own increasing index ranges and each rank's
candidates arrive sorted by (score desc, index asc), so the candidates'
positions in the gathered array order equal scores by global move index, the
tie rule of the single-GPU selection.

Host plumbing only; every score, flag and selection comes from the CUDA
library.  ``torch.distributed`` carries the exchange (NCCL on GPUs; the gloo
backend on the CPU in the tests, where the evaluation is supplied by the
caller).
"""

from __future__ import annotations

from typing import Callable, Tuple

import numpy as np


def shard_range(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous slice [lo, hi) of n moves owned by rank (sizes differ by at
    most one; every move belongs to exactly one rank)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard request n={n} world={world} rank={rank}")
    return n * rank // world, n * (rank + 1) // world


def gather_candidates(idx_local, top_local, count_local: int, lo: int, k: int, group=None):
    """All-gather every rank's top-k keys.

    idx_local[k] (int32, indices within the rank's slice), top_local[k]
    (float32) and count_local describe the rank's selection; lo is the slice's
    first global index.  Returns (cand_idx int64[world*k] of global move
    indices, cand_score float32[world*k], cand_flag uint8[world*k] = 1 for
    the first count entries of each rank), in rank order, as tensors on the
    device of idx_local."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = idx_local.device
    gidx = torch.full((k,), -1, dtype=torch.int64, device=dev)
    gsc = torch.zeros(k, dtype=torch.float32, device=dev)
    c = int(count_local)
    if c > 0:
        gidx[:c] = idx_local[:c].to(torch.int64) + lo
        gsc[:c] = top_local[:c]
    cnt = torch.tensor([c], dtype=torch.int64, device=dev)
    all_idx = [torch.empty_like(gidx) for _ in range(world)]
    all_sc = [torch.empty_like(gsc) for _ in range(world)]
    all_cnt = [torch.empty_like(cnt) for _ in range(world)]
    dist.all_gather(all_idx, gidx, group=group)
    dist.all_gather(all_sc, gsc, group=group)
    dist.all_gather(all_cnt, cnt, group=group)
    flag = torch.zeros(world * k, dtype=torch.uint8, device=dev)
    for r in range(world):
        flag[r * k: r * k + int(all_cnt[r].item())] = 1
    return torch.cat(all_idx), torch.cat(all_sc), flag


def sharded_topk(local_select: Callable[[int, int], tuple], merge_select: Callable, n: int, k: int, group=None):
    """The batch's top k over ranks.

    local_select(lo, hi) evaluates moves [lo, hi) of the batch and returns the
    slice's (idx, top, count) top-k selection (indices within the slice);
    merge_select(score, flag, k) selects from the gathered candidates and
    returns (positions, scores, count).  Returns (global move indices int64,
    scores float32, count) identical on every rank."""
    import torch.distributed as dist

    world, rank = dist.get_world_size(group), dist.get_rank(group)
    lo, hi = shard_range(n, world, rank)
    idx, top, cnt = local_select(lo, hi)
    cidx, csc, cflag = gather_candidates(idx, top, int(cnt), lo, k, group)
    pos, sc, c = merge_select(csc, cflag, k)
    c = int(c)
    return cidx[pos[:c].long()], sc[:c], c


def model_sharded_topk(model, moves_dev, k: int, group=None):
    """sharded_topk with the CUDA library on each rank's GPU: mm_eval_moves
    and mm_topk on the rank's slice, then mm_topk over the candidates."""
    import torch

    n = int(moves_dev.shape[0])

    def local(lo, hi):
        s, f, _ = model.eval_moves(moves_dev[lo:hi], want_mean=False)
        i, t, c = model.topk(s, f, k)
        return i, t, int(c.cpu()[0])

    def merge(score, flag, kk):
        i, t, c = model.topk(score.contiguous(), flag.contiguous(), kk)
        return i, t, int(c.cpu()[0])

    return sharded_topk(local, merge, n, k, group)
