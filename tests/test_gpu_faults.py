"""Failure handling without any GPU fault: invalid arguments are refused on
the host with MM_ERR_INVALID_ARG / MM_ERR_STATE; a corrupted move list is
flagged (flag 0, score -inf, sticky MM_ERR_BAD_MOVE on the next synchronising
call) and leaves the model usable; an allocation cap (host-side injection,
MM_ALLOC_CAP_BYTES) turns model creation into MM_ERR_OOM with nothing left
allocated; a bounded device wait made to run out (test-only mode, set at
model creation: the bulk-copy stages expect bytes that never come, every copy
issued still lands; or the relaxed forward's stage barriers expect one
arrival that never comes) returns MM_ERR_TIMEOUT at the next synchronising
call and leaves the model usable.  Nothing here traps, faults or hangs the
GPU."""

import ctypes as C
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

INVALID_ARG, OOM, BAD_MOVE, TIMEOUT, STATE = 1, 3, 6, 7, 8


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _mm():
    import paper_2511_18296_b300 as mm
    return mm


def test_invalid_arguments_refused_on_the_host():
    mm = _mm()
    L = mm.lib()
    p = W.config("plain_4k")
    m = mm.Model.from_problem(p)
    n = p.moves.shape[0]
    mv = torch.as_tensor(p.moves, device="cuda")
    score = torch.empty(n, device="cuda")
    feas = torch.empty(n, dtype=torch.uint8, device="cuda")
    # no schedule installed yet
    assert L.mm_eval_moves(m.h, mv.data_ptr(), n, score.data_ptr(), feas.data_ptr(), None) == STATE
    m.schedule_set(p.x0)
    assert L.mm_eval_moves(None, mv.data_ptr(), n, score.data_ptr(), feas.data_ptr(), None) == INVALID_ARG
    assert L.mm_eval_moves(m.h, mv.data_ptr(), -1, score.data_ptr(), feas.data_ptr(), None) == INVALID_ARG
    assert L.mm_eval_moves(m.h, mv.data_ptr() + 4, n - 1, score.data_ptr(), feas.data_ptr(), None) == INVALID_ARG
    assert L.mm_eval_moves(m.h, None, n, score.data_ptr(), feas.data_ptr(), None) == INVALID_ARG
    idx = torch.empty(32, dtype=torch.int32, device="cuda")
    top = torch.empty(32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    for k in (0, 1025):
        assert L.mm_topk(m.h, score.data_ptr(), feas.data_ptr(), n, k, idx.data_ptr(), top.data_ptr(),
                         cnt.data_ptr()) == INVALID_ARG
    bad = p.x0.copy()
    bad[0] = p.T + 1
    assert L.mm_schedule_set(m.h, bad.ctypes.data, None) == INVALID_ARG
    assert L.mm_last_error().decode()  # a message explains each refusal
    # the model still works
    s1, f1, _ = m.eval_moves(mv, want_mean=False)
    torch.cuda.synchronize()
    assert f1.cpu().numpy().sum() > 0


def test_corrupted_move_list_is_flagged_and_the_model_stays_usable():
    mm = _mm()
    p = W.config("plain_4k")
    m = mm.Model.from_problem(p)
    m.schedule_set(p.x0)
    rng = np.random.default_rng(13)
    junk = rng.integers(-2**31, 2**31 - 1, size=(5000, 2), dtype=np.int64).astype(np.int32)
    junk[:10] = p.moves[:10]  # a few genuine moves among the garbage
    s, f, _ = m.eval_moves(torch.as_tensor(junk, device="cuda"), want_mean=False)
    torch.cuda.synchronize()
    s, f = s.cpu().numpy(), f.cpu().numpy()
    valid = (junk[:, 0] >= 0) & (junk[:, 0] < p.B) & (((junk[:, 1] >= 0) & (junk[:, 1] < p.B)) |
                                                     ((junk[:, 1] < 0) & (junk[:, 1] >= -(p.T + 1))))
    assert np.all(f[~valid] == 0) and np.all(np.isneginf(s[~valid]))
    with pytest.raises(mm.MMError) as e:
        m.npv()
    assert e.value.status == BAD_MOVE
    # cleared by the read: the same model evaluates the genuine batch as a fresh one does
    fresh = mm.Model.from_problem(p)
    fresh.schedule_set(p.x0)
    mv = torch.as_tensor(p.moves, device="cuda")
    a = m.eval_moves(mv, want_mean=False)[0].cpu().numpy()
    b = fresh.eval_moves(mv, want_mean=False)[0].cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    m.npv()  # no sticky status left


def test_allocation_cap_gives_out_of_memory():
    mm = _mm()
    p = W.config("plain_4k")
    os.environ["MM_ALLOC_CAP_BYTES"] = "100000"  # the 4k model's FP64 grade array alone is 4,000 x 16 x 8 = 512,000 bytes
    try:
        with pytest.raises(mm.MMError) as e:
            mm.Model.from_problem(p)
        assert e.value.status == OOM
    finally:
        del os.environ["MM_ALLOC_CAP_BYTES"]
    m = mm.Model.from_problem(p)  # without the cap the same model is created and works
    m.schedule_set(p.x0)
    m.npv()


def test_bulk_copy_wait_runs_out_and_the_model_stays_usable(monkeypatch):
    """With MM_TEST_STALL_BULK_WAIT set at model creation every stage of the
    bulk-copy evaluator expects 16 bytes that no copy delivers, so its bounded
    wait (about 1 ms in this mode) runs out; the warp then waits, bounded
    again, for the copies it issued (they all land) and leaves.  The next
    synchronising call reports MM_ERR_TIMEOUT once; the same model then
    evaluates the batch with direct loads, matching the FP64 oracle."""
    import oracle as O
    from helpers import assert_close_floor
    mm = _mm()
    p = W.config("plain_4k", n_moves=1024)
    monkeypatch.setenv("MM_TEST_STALL_BULK_WAIT", "1")
    m = mm.Model.from_problem(p)
    monkeypatch.delenv("MM_TEST_STALL_BULK_WAIT")
    m.schedule_set(p.x0)
    mv = torch.as_tensor(p.moves, device="cuda")
    m.set_tile(stages=2)  # the bulk-copy evaluator
    m.eval_moves(mv, want_mean=False)
    with pytest.raises(mm.MMError) as e:
        m.npv()
    assert e.value.status == TIMEOUT
    m.npv()  # reported once, then cleared
    m.set_tile(stages=0)  # direct loads: no bulk copies, no waits
    s, f, _ = m.eval_moves(mv, want_mean=False)
    torch.cuda.synchronize()
    ref = O.OracleModel(p).eval_incremental(p.x0, p.moves)
    assert np.array_equal(f.cpu().numpy(), ref["flag"])
    assert_close_floor(s.cpu().numpy(), ref["score"], ref["floor"], what="scores after the timeout")
    m.npv()


def test_relaxed_forward_wait_runs_out_and_the_model_stays_usable(monkeypatch):
    """With MM_TEST_STALL_RELAXED set at model creation the next relaxed
    forward's stage barriers expect one arrival that no thread makes, and
    every wait of that launch gives up after about 1 ms: the copy warps wait
    for their copies (they all land), no product is issued, the tensor memory
    is released.  The next synchronising call reports MM_ERR_TIMEOUT once; the
    mode is one-shot, so the same model's next forward matches the float64
    oracle."""
    mm = _mm()
    from test_gpu_relaxed import TOL, reference
    from helpers import tiny_problem
    p = tiny_problem(8, 8, 4, S=100, T=20, seed=11, target_blocks=8)
    x = W.relaxed_x(p.B, p.T, 2)
    g = p.grade.astype(np.float32)
    monkeypatch.setenv("MM_TEST_STALL_RELAXED", "1")
    m = mm.Model.from_problem(p)
    monkeypatch.delenv("MM_TEST_STALL_RELAXED")
    m.schedule_set(p.x0)  # for the synchronising npv calls below
    xt = torch.as_tensor(x, device="cuda")
    gt = torch.as_tensor(g, device="cuda")
    m.relaxed_forward(xt, gt)
    with pytest.raises(mm.MMError) as e:
        m.npv()
    assert e.value.status == TIMEOUT
    m.npv()  # reported once, then cleared
    J, npv, ot = m.relaxed_forward(xt, gt)
    torch.cuda.synchronize()
    r = reference(p, x, g)
    assert float(J.cpu()[0]) == pytest.approx(r["J"], rel=TOL)
    np.testing.assert_allclose(npv.cpu().numpy(), r["npv"], rtol=TOL)
    m.npv()
