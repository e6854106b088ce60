"""The multi-rank path on the CPU: two gloo ranks (world size 2, 127.0.0.1).

paper_2511_18296_b300.dist splits a batch of moves into contiguous slices,
one per rank, all-gathers each rank's top k and merges them.  Here each rank's
evaluation and both selections come from the FP64 oracle (there is no GPU on
this machine); what is tested is the host logic: the slices, the global
indices, the exchange and the exactness of the merge, including ties across
the slice boundary.  The result must equal the single-process selection over
the whole batch bit for bit.
"""

import os
import socket

import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2511_18296_b300 import dist as D

K = 32


def test_shard_range_partitions_every_batch():
    for n in (0, 1, 5, 7, 4096, 262144):
        for world in (1, 2, 3, 5, 8):
            seen = []
            for r in range(world):
                lo, hi = D.shard_range(n, world, r)
                assert 0 <= lo <= hi <= n
                assert hi - lo in (n // world, n // world + 1)
                seen.extend(range(lo, hi))
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        D.shard_range(10, 2, 2)


def _scores(kind):
    """Scores and flags of the whole batch: the oracle's on the 4k workload,
    or a tie-heavy synthetic set (few distinct values, ties across ranks)."""
    p = W.config("plain_4k")
    if kind == "oracle":
        r = O.OracleModel(p).eval_incremental(p.x0, p.moves)
        return r["score"].astype(np.float32), r["flag"].astype(np.uint8)
    n = p.moves.shape[0]
    i = np.arange(n)
    s = ((i * 7919) % 5).astype(np.float32) - 2.0  # five values, each shared by ~800 moves
    s[(i % 97) == 0] = 0.0
    s[(i % 89) == 0] = -0.0
    f = ((i % 3) != 0).astype(np.uint8)
    return s, f


def _worker(rank, world, port, kind, out_path):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, f = _scores(kind)

        def local(lo, hi):
            idx, top = O.topk(s[lo:hi], f[lo:hi], K)
            i = torch.zeros(K, dtype=torch.int32)
            t = torch.zeros(K, dtype=torch.float32)
            i[:len(idx)] = torch.from_numpy(idx.astype(np.int32))
            t[:len(top)] = torch.from_numpy(top.astype(np.float32))
            return i, t, len(idx)

        def merge(score, flag, k):
            pos, top = O.topk(score.numpy(), flag.numpy(), k)
            return torch.from_numpy(pos.astype(np.int64)), torch.from_numpy(top.astype(np.float32)), len(pos)

        gi, gs, c = D.sharded_topk(local, merge, s.shape[0], K)
        np.savez(out_path, idx=gi.numpy(), score=gs.numpy(), count=c)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("kind", ["oracle", "ties"])
def test_two_gloo_ranks_merge_exactly(tmp_path, kind):
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    outs = [str(tmp_path / f"rank{r}.npz") for r in range(world)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, outs[r])) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0, f"rank exited with {pr.exitcode}"
    s, f = _scores(kind)
    ref_idx, ref_top = O.topk(s, f, K)
    for o in outs:
        r = np.load(o)
        assert int(r["count"]) == len(ref_idx)
        assert np.array_equal(r["idx"], ref_idx.astype(np.int64))
        assert np.array_equal(r["score"], ref_top.astype(np.float32))


def _step_worker(rank, world, port, steps, out_path):
    """A sharded search step per iteration: the rank evaluates its slice of
    the batch on its own replica of the schedule (the oracle stands in for the
    GPU), the ranks exchange their top k, and every rank applies the winner to
    its replica."""
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = W.config("plain_4k")
        om = O.OracleModel(p)
        x = p.x0.copy()

        def local(lo, hi):
            r = om.eval_incremental(x, p.moves[lo:hi])
            idx, top = O.topk(r["score"].astype(np.float32).astype(np.float64), r["flag"], K)
            i = torch.zeros(K, dtype=torch.int32)
            t = torch.zeros(K, dtype=torch.float32)
            i[:len(idx)] = torch.from_numpy(idx.astype(np.int32))
            t[:len(top)] = torch.from_numpy(top.astype(np.float32))
            return i, t, len(idx)

        def merge(score, flag, k):
            pos, top = O.topk(score.numpy().astype(np.float64), flag.numpy(), k)
            return torch.from_numpy(pos.astype(np.int64)), torch.from_numpy(top.astype(np.float32)), len(pos)

        def apply_winner(g):
            assert om.apply(x, p.moves[g]) == 0

        winners = []
        for _ in range(steps):
            gi, gs, c = D.sharded_step(local, merge, apply_winner, p.moves.shape[0], K)
            winners.append(int(gi[0]) if c else -1)
        np.savez(out_path, x=x, npv=om.npv(x), winners=np.asarray(winners))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharded_steps_keep_replicas_identical(tmp_path):
    """24 sharded steps on two ranks: both replicas end with the same schedule
    and bit-identical FP64 NPV, and every step applied the move a single
    process selects over the whole batch (same FP32-rounded scores)."""
    import torch.multiprocessing as mp

    world, steps = 2, 24
    port = _free_port()
    outs = [str(tmp_path / f"step{r}.npz") for r in range(world)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_step_worker, args=(r, world, port, steps, outs[r])) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(300)
        assert pr.exitcode == 0, f"rank exited with {pr.exitcode}"
    res = [np.load(o) for o in outs]
    assert np.array_equal(res[0]["x"], res[1]["x"])
    assert np.array_equal(res[0]["npv"].view(np.uint64), res[1]["npv"].view(np.uint64))
    assert np.array_equal(res[0]["winners"], res[1]["winners"])
    # the single-process reference: the whole batch, the same steps
    p = W.config("plain_4k")
    om = O.OracleModel(p)
    x = p.x0.copy()
    ref = []
    for _ in range(steps):
        r = om.eval_incremental(x, p.moves)
        idx, _ = O.topk(r["score"].astype(np.float32).astype(np.float64), r["flag"], K)
        ref.append(int(idx[0]) if len(idx) else -1)
        if len(idx):
            assert om.apply(x, p.moves[idx[0]]) == 0
    assert np.array_equal(res[0]["winners"], np.asarray(ref))
    assert np.array_equal(res[0]["x"], x)
    assert (np.asarray(ref) >= 0).sum() == steps  # every step applied a move
