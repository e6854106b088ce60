"""Several GPUs, one process each: the batch of moves split across ranks.

Moves are independent once the block model and the schedule are fixed, so a
batch partitions into contiguous slices, one per rank, with move indices kept
global.  Each rank evaluates its slice and selects its own top k; the only
exchange is an all-gather of the ranks' k (index, score) keys, after which
every rank selects the batch's top k from the gathered candidates with the
library's top-k kernel and applies the same best move to its replica of the
state (Algorithm 4's assignment after Algorithm 5's evaluation), so all
replicas stay identical, FP64 totals included: every replica runs the same
deterministic apply on the same state.  Per step a rank sends k keys of 12
bytes (8-byte index, 4-byte score) and an 8-byte count.  (When every rank
searches its own independent batch, nothing is exchanged at all.)

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


def sharded_step(local_select: Callable[[int, int], tuple], merge_select: Callable,
                 apply_winner: Callable[[int], None], n: int, k: int, group=None):
    """One search step over ranks: sharded_topk, then apply_winner(global
    index of the batch's best move) on this rank's replica when some move is
    feasible.  Every rank applies the same move.  Returns what sharded_topk
    returns."""
    gi, gs, c = sharded_topk(local_select, merge_select, n, k, group)
    if c > 0:
        apply_winner(int(gi[0]))
    return gi, gs, c


def model_sharded_step(model, moves_dev, k: int, group=None):
    """sharded_step with the CUDA library, without a host round trip: the
    fused step on the rank's slice with apply off (mm_search_step), an
    all-gather of the k keys and the count (device tensors), the exact merge
    (mm_topk over the candidates), then the device apply of the best move
    (mm_apply_best on the whole batch with its global index).  Returns (global
    move indices int64 [k], scores float32 [k], count int32 [1]), device
    tensors equal on every rank; entries past the count are unspecified."""
    import torch
    import torch.distributed as dist

    n = int(moves_dev.shape[0])
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    lo, hi = shard_range(n, world, rank)
    dev = moves_dev.device
    _, _, idx, top, cnt = model.search_step(moves_dev[lo:hi], k=k, apply=False)
    live = torch.arange(k, device=dev) < cnt.to(torch.int64)
    gidx = torch.where(live, idx.to(torch.int64) + lo, torch.full_like(idx, -1, dtype=torch.int64))
    gsc = torch.where(live, top, torch.zeros_like(top))
    all_idx = [torch.empty_like(gidx) for _ in range(world)]
    all_sc = [torch.empty_like(gsc) for _ in range(world)]
    all_cnt = [torch.empty_like(cnt) for _ in range(world)]
    dist.all_gather(all_idx, gidx, group=group)
    dist.all_gather(all_sc, gsc, group=group)
    dist.all_gather(all_cnt, cnt, group=group)
    cidx, csc = torch.cat(all_idx), torch.cat(all_sc)
    cnts = torch.cat(all_cnt).to(torch.int64)
    cflag = (torch.arange(k, device=dev)[None, :] < cnts[:, None]).reshape(-1).to(torch.uint8)
    pos, best, count = model.topk(csc.contiguous(), cflag.contiguous(), k)
    # positions past the count are unspecified: clamp before the gather
    gpos = pos.to(torch.int64).clamp(0, world * k - 1)
    win = cidx[gpos]
    model.apply_best(moves_dev, win[:1].to(torch.int32).contiguous(), count)
    return win, best, count
