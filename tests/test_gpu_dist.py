"""The multi-rank top-k path with the CUDA library (one GPU).

One process can hold one GPU only, so the rank exchange runs as a world of one
(NCCL) through model_sharded_topk, and the merge of several slices' top k is
checked by hand: slices evaluated and selected separately by the library,
their candidates laid out as the all-gather would, and selected again by the
library, must give the single-launch selection over the whole batch.
"""

import os
import socket

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = 32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _model(name, n_moves=None):
    import paper_2511_18296_b300 as mm
    p = W.config(name, n_moves=n_moves)
    m = mm.Model.from_problem(p)
    assert m.schedule_set(p.x0)
    return p, m, torch.as_tensor(p.moves, device="cuda")


@pytest.mark.parametrize("slices", [2, 3, 7])
def test_slice_topk_merge_equals_whole_batch(slices):
    from paper_2511_18296_b300 import dist as D
    p, m, mv = _model("plain_50k", n_moves=65536)
    n = mv.shape[0]
    s, f, _ = m.eval_moves(mv, want_mean=False)
    ref_i, ref_t, ref_c = m.topk(s, f, K)
    cidx, csc, cfl = [], [], []
    for r in range(slices):
        lo, hi = D.shard_range(n, slices, r)
        ls, lf, _ = m.eval_moves(mv[lo:hi], want_mean=False)
        assert torch.equal(ls, s[lo:hi]) and torch.equal(lf, f[lo:hi])
        i, t, c = m.topk(ls, lf, K)
        c = int(c.cpu()[0])
        gi = torch.full((K,), -1, dtype=torch.int64, device="cuda")
        gi[:c] = i[:c].long() + lo
        gs = torch.zeros(K, device="cuda")
        gs[:c] = t[:c]
        fl = torch.zeros(K, dtype=torch.uint8, device="cuda")
        fl[:c] = 1
        cidx.append(gi), csc.append(gs), cfl.append(fl)
    cidx, csc, cfl = torch.cat(cidx), torch.cat(csc), torch.cat(cfl)
    pos, top, cnt = m.topk(csc, cfl, K)
    c = int(cnt.cpu()[0])
    assert c == int(ref_c.cpu()[0])
    assert torch.equal(cidx[pos[:c].long()].cpu(), ref_i[:c].long().cpu())
    assert torch.equal(top[:c].cpu(), ref_t[:c].cpu())


def test_world_of_one_nccl():
    import torch.distributed as dist
    from paper_2511_18296_b300 import dist as D
    p, m, mv = _model("plain_4k")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        gi, gs, c = D.model_sharded_topk(m, mv, K)
    finally:
        dist.destroy_process_group()
    s, f, _ = m.eval_moves(mv, want_mean=False)
    ri, rt, rc = m.topk(s, f, K)
    assert c == int(rc.cpu()[0])
    assert torch.equal(gi.cpu(), ri[:c].long().cpu())
    assert torch.equal(gs.cpu(), rt[:c].cpu())


def test_sharded_steps_keep_replicas_equal_to_one_model():
    """Two replicas of the model, each evaluating one slice of the batch with
    the fused step (apply off); their top k laid out as the all-gather would,
    merged by the library, and the winner applied on both replicas by the
    device apply: over 8 steps both replicas stay equal to a single model that
    runs the fused step with apply on the whole batch (top k, schedule and
    NPV bit for bit)."""
    import paper_2511_18296_b300 as mm
    from paper_2511_18296_b300 import dist as D
    p = W.config("plain_50k", n_moves=65536)
    reps = [mm.Model.from_problem(p) for _ in range(2)]
    one = mm.Model.from_problem(p)
    for m in reps + [one]:
        m.schedule_set(p.x0)
    mv = torch.as_tensor(p.moves, device="cuda")
    n = mv.shape[0]
    for _ in range(8):
        cands = []
        for r, m in enumerate(reps):
            lo, hi = D.shard_range(n, 2, r)
            _, _, i, t, c = m.search_step(mv[lo:hi], k=K, apply=False)
            live = torch.arange(K, device="cuda") < c.long()
            cands.append((torch.where(live, i.long() + lo, -1), torch.where(live, t, 0.0), c))
        cidx = torch.cat([x[0] for x in cands])
        csc = torch.cat([x[1] for x in cands])
        cfl = torch.cat([(torch.arange(K, device="cuda") < x[2].long()).to(torch.uint8) for x in cands])
        win = []
        for m in reps:  # every replica merges the same candidates and applies the winner
            pos, top, cnt = m.topk(csc, cfl, K)
            g = cidx[pos.long().clamp(0, 2 * K - 1)]
            m.apply_best(mv, g[:1].int().contiguous(), cnt)
            win.append((g, top, cnt))
        _, _, oi, ot, oc = one.search_step(mv, k=K, apply=True)
        torch.cuda.synchronize()
        c = int(oc.cpu()[0])
        for g, top, cnt in win:
            assert int(cnt.cpu()[0]) == c
            assert torch.equal(g[:c].cpu(), oi[:c].long().cpu())
            assert torch.equal(top[:c].cpu(), ot[:c].cpu())
    x1 = one.schedule_get()
    for m in reps:
        assert np.array_equal(m.schedule_get(), x1)
        assert np.array_equal(m.npv()[0], one.npv()[0])


def test_model_sharded_step_world_of_one():
    import torch.distributed as dist
    from paper_2511_18296_b300 import dist as D
    import paper_2511_18296_b300 as mm
    p = W.config("plain_4k")
    a = mm.Model.from_problem(p)
    b = mm.Model.from_problem(p)
    a.schedule_set(p.x0)
    b.schedule_set(p.x0)
    mv = torch.as_tensor(p.moves, device="cuda")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        for _ in range(5):
            gi, gs, gc = D.model_sharded_step(a, mv, K)
            _, _, bi, bt, bc = b.search_step(mv, k=K, apply=True)
            torch.cuda.synchronize()
            c = int(bc.cpu()[0])
            assert int(gc.cpu()[0]) == c
            assert torch.equal(gi[:c].cpu(), bi[:c].long().cpu())
            assert torch.equal(gs[:c].cpu(), bt[:c].cpu())
    finally:
        dist.destroy_process_group()
    assert np.array_equal(a.schedule_get(), b.schedule_get())
    assert np.array_equal(a.npv()[0], b.npv()[0])
