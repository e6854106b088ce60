"""Fused search step (mm_search_step) vs the separate calls it fuses.

One launch evaluates the batch, keeps each warp's best 32 keys with warp
shuffles, merges them at the end of the launch and applies the best move.
It must reproduce mm_eval_moves + mm_topk + mm_apply_best exactly: same scores
and flags bit for bit, same top-k, same schedule and NPV after every step.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import all_moves, tiny_problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _pair(p):
    import paper_2511_18296_b300 as mm
    a = mm.Model.from_problem(p)
    b = mm.Model.from_problem(p)
    a.schedule_set(p.x0)
    b.schedule_set(p.x0)
    return a, b


def _separate(m, mv, k, apply):
    s, f, _ = m.eval_moves(mv, want_mean=False)
    idx, top, cnt = m.topk(s, f, k)
    if apply:
        m.apply_best(mv, idx, cnt)
    return s, f, idx, top, cnt


def _compare(ra, rb, k):
    torch.cuda.synchronize()
    sa, fa, ia, ta, ca = (x.cpu().numpy() for x in ra)
    sb, fb, ib, tb, cb = (x.cpu().numpy() for x in rb)
    assert np.array_equal(fa, fb)
    assert np.array_equal(sa.view(np.uint32), sb.view(np.uint32))
    assert ca[0] == cb[0]
    c = int(ca[0])
    assert np.array_equal(ia[:c], ib[:c]) and np.array_equal(ta[:c], tb[:c])
    return c


@pytest.mark.parametrize("name,steps,k", [("plain_4k", 12, 32), ("plain_50k", 4, 8)])
def test_step_matches_separate_calls(name, steps, k):
    p = W.config(name)
    a, b = _pair(p)
    mv = torch.as_tensor(p.moves, device="cuda")
    for _ in range(steps):
        ra = a.search_step(mv, k=k, apply=True)
        rb = _separate(b, mv, k, True)
        _compare(ra, rb, k)
        la, lb = a.last_apply(), b.last_apply()
        assert la == lb
    assert np.array_equal(a.schedule_get(), b.schedule_get())
    na, nb = a.npv(), b.npv()
    assert np.array_equal(na[0], nb[0])


@pytest.mark.parametrize("n", [1, 63, 64, 65, 1000, 20_000])
@pytest.mark.parametrize("k", [1, 7, 32])
def test_step_sizes_and_k(n, k):
    p = W.config("plain_4k", n_moves=max(n, 2))
    a, b = _pair(p)
    mv = torch.as_tensor(p.moves[:n], device="cuda")
    ra = a.search_step(mv, k=k, apply=False)
    rb = _separate(b, mv, k, False)
    c = _compare(ra, rb, k)
    # no apply: the schedule is unchanged
    assert np.array_equal(a.schedule_get(), p.x0)
    # and the selection is the oracle's on the GPU's own scores
    s, f = ra[0].cpu().numpy(), ra[1].cpu().numpy()
    ri, _ = O.topk(s.astype(np.float64), f, k)
    assert np.array_equal(ra[2].cpu().numpy()[:c], ri)


def test_step_run_time_shaped_loop():
    """S = 13 (not a multiple of 4) runs the run-time-shaped evaluator."""
    p = tiny_problem(3, 3, 3, S=13, T=3, seed=4)
    a, b = _pair(p)
    mv = torch.as_tensor(all_moves(p.B, p.T), device="cuda")
    for _ in range(3):
        _compare(a.search_step(mv, k=5, apply=True), _separate(b, mv, 5, True), 5)
    assert np.array_equal(a.schedule_get(), b.schedule_get())


def test_step_nothing_feasible_and_errors():
    import paper_2511_18296_b300 as mm
    p = W.config("plain_4k")
    a, _ = _pair(p)
    inc = O.OracleModel(p).eval_incremental(p.x0, p.moves)
    bad = torch.as_tensor(p.moves[inc["flag"] == 0][:500], device="cuda")
    s, f, idx, top, cnt = a.search_step(bad, k=4, apply=True)
    torch.cuda.synchronize()
    assert int(cnt.cpu()[0]) == 0
    assert a.last_apply()[0] == 0
    assert np.array_equal(a.schedule_get(), p.x0)
    with pytest.raises(mm.MMError):
        a.search_step(bad, k=33)


def test_step_event_splits_the_two_launches():
    """The timing hook records the caller's event between the evaluation and
    the apply launch, eagerly and as an external node of a captured graph; the
    step's results do not change."""
    p = W.config("plain_4k")
    a, b = _pair(p)
    st = torch.cuda.Stream()
    a.set_stream(st)
    mv = torch.as_tensor(p.moves, device="cuda")
    out = [torch.empty(p.moves.shape[0], device="cuda"), torch.empty(p.moves.shape[0], dtype=torch.uint8, device="cuda"),
           torch.empty(32, dtype=torch.int32, device="cuda"), torch.empty(32, device="cuda"),
           torch.empty(1, dtype=torch.int32, device="cuda")]
    mid = torch.cuda.Event(enable_timing=True)
    with pytest.raises(ValueError):
        a.set_step_event(mid)  # not recorded yet: no handle
    mid.record(st)
    a.set_step_event(mid)

    def step():
        a.search_step(mv, k=32, apply=True, score=out[0], feas=out[1], idx=out[2], top=out[3], count=out[4])

    with torch.cuda.stream(st):
        step()  # eager
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        step()
    a.set_step_event(None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        e0.record(st)
        g.replay()
        e1.record(st)
    e1.synchronize()
    t_eval, t_fin = e0.elapsed_time(mid), mid.elapsed_time(e1)
    assert t_eval > 0 and t_fin > 0 and t_eval + t_fin == pytest.approx(e0.elapsed_time(e1), rel=1e-3, abs=1e-3)
    # two steps through the hook agree with two plain steps
    for _ in range(2):
        rb = b.search_step(mv, k=32, apply=True)
    _compare(out, rb, 32)
    assert np.array_equal(a.schedule_get(), b.schedule_get())


@pytest.mark.parametrize("name,steps", [("plain_4k", 60), ("plain_50k", 30)])
def test_step_state_matches_rebuild(name, steps):
    """After every fused step, the running FP64 state (per-period tonnage,
    metal, NPV_s) equals a from-scratch rebuild of the same schedule on a
    fresh model: exactly for the integer tonnages, to FP64 rounding for the
    metal and NPV.  Many steps, so an ordering race inside the in-launch apply
    (one thread updating a value others still read) cannot hide."""
    p = W.config(name)
    a, fresh = _pair(p)
    mv = torch.as_tensor(p.moves, device="cuda")
    for _ in range(steps):
        a.search_step(mv, k=8, apply=True)
        assert a.last_apply()[0] == 1
        fresh.schedule_set(a.schedule_get())
        ma, oa = a.tonnage()
        mf, of = fresh.tonnage()
        assert np.array_equal(ma, mf) and np.array_equal(oa, of)
        np.testing.assert_allclose(a.metal(), fresh.metal(), rtol=1e-12, atol=1e-6)
        npv_a, npv_f = a.npv()[0], fresh.npv()[0]
        np.testing.assert_allclose(npv_a, npv_f, rtol=1e-12, atol=1e-3)


def test_step_run_time_shaped_loop_large_tables():
    """S = 101 (not a multiple of 4), T = 30: the run-time-shaped step kernel
    with its penalty tables staged in shared memory (25.8 KB) on top of the
    in-launch apply's static buffers, past the 48 KB default."""
    p = tiny_problem(8, 8, 4, S=101, T=30, seed=6, cap_blocks=12, target_blocks=5)
    a, b = _pair(p)
    mv = torch.as_tensor(all_moves(p.B, p.T)[::7].copy(), device="cuda")
    for _ in range(3):
        _compare(a.search_step(mv, k=8, apply=True), _separate(b, mv, 8, True), 8)
    assert np.array_equal(a.schedule_get(), b.schedule_get())


def test_step_fp64_update_settles_before_every_reader():
    """The fused step's final CTA applies the structural part of the best move
    (tonnage, schedule words, tables) and leaves its FP64 part (metal, net
    cash, NPV_s) to the first CTA of the next step, or to the library before
    any call that reads or changes those totals.  Interleave fused steps with
    each such call on one model and the separate calls on a twin: every
    result must be the same bits.  Batches of 100 moves run as one CTA (its
    first and final CTA are the same)."""
    import paper_2511_18296_b300 as mm
    p = W.config("plain_4k")
    a, b = _pair(p)
    mv = torch.as_tensor(p.moves, device="cuda")
    small = torch.as_tensor(p.moves[:100], device="cuda")

    def both_step(batch, k=8):
        _compare(a.search_step(batch, k=k, apply=True), _separate(b, batch, k, True), k)

    def same_npv():
        na, nb = a.npv(), b.npv()
        assert np.array_equal(na[0], nb[0]) and na[1:] == nb[1:]

    both_step(mv)
    same_npv()                                   # mm_npv settles
    both_step(mv)
    both_step(small)                             # one CTA: first finisher and final CTA at once
    assert a.last_apply() == b.last_apply()      # mm_last_apply settles
    both_step(mv)
    assert np.array_equal(a.metal(), b.metal())  # mm_get_metal settles
    both_step(mv)
    inc = O.OracleModel(p).eval_incremental(a.schedule_get(), p.moves)
    j = int(np.flatnonzero(inc["flag"])[0])
    assert a.apply_move(tuple(p.moves[j])) == b.apply_move(tuple(p.moves[j]))  # mm_apply_move settles first
    same_npv()
    for m in (a, b):
        m.set_fp32_shadow(True)                  # the shadow starts from settled totals
    both_step(mv)
    both_step(mv)
    assert np.array_equal(a.fp32_shadow_npv(), b.fp32_shadow_npv())
    for m in (a, b):
        m.set_fp32_shadow(False)
    both_step(mv)
    for m in (a, b):                             # a batch that applies settles its chains first
        bt = mm.Batch([(m, small)], k=4, apply=True)
        bt.run()
        torch.cuda.synchronize()
        bt.close()
    same_npv()
    both_step(mv)                                # a new schedule voids the update still due
    for m in (a, b):
        m.schedule_set(p.x0)
    same_npv()
    both_step(mv)
    st = torch.cuda.Stream()                     # steps replayed from a captured graph
    a.set_stream(st)
    outs = [torch.empty(p.moves.shape[0], device="cuda"), torch.empty(p.moves.shape[0], dtype=torch.uint8,
            device="cuda"), torch.empty(8, dtype=torch.int32, device="cuda"), torch.empty(8, device="cuda"),
            torch.empty(1, dtype=torch.int32, device="cuda")]
    step = lambda: a.search_step(mv, k=8, apply=True, score=outs[0], feas=outs[1], idx=outs[2], top=outs[3],  # noqa
                                 count=outs[4])
    with torch.cuda.stream(st):
        step()
    st.synchronize()
    _separate(b, mv, 8, True)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        step()
        step()
    for _ in range(3):
        g.replay()
        for _ in range(2):
            rb = _separate(b, mv, 8, True)
    st.synchronize()
    _compare(outs, rb, 8)
    assert np.array_equal(a.schedule_get(), b.schedule_get())
    same_npv()


@pytest.mark.parametrize("S", [260, 500, 768])
def test_step_in_launch_apply_up_to_768_scenarios(S):
    """Up to 768 scenarios (one thread each in the step's CTA) the best move is
    applied inside the step's launch: same scores, flags, top-k, schedule and
    NPV as the separate calls, and the FP64 state equals a rebuild."""
    p = tiny_problem(6, 6, 3, S=S, T=6, seed=S, cap_blocks=8, target_blocks=3)
    a, b = _pair(p)
    mv = torch.as_tensor(all_moves(p.B, p.T)[::3].copy(), device="cuda")
    for _ in range(4):
        _compare(a.search_step(mv, k=8, apply=True), _separate(b, mv, 8, True), 8)
        assert a.last_apply() == b.last_apply()
    assert np.array_equal(a.schedule_get(), b.schedule_get())
    assert np.array_equal(a.npv()[0], b.npv()[0])
    import paper_2511_18296_b300 as mm
    fresh = mm.Model.from_problem(p)
    fresh.schedule_set(a.schedule_get())
    np.testing.assert_allclose(a.npv()[0], fresh.npv()[0], rtol=1e-12, atol=1e-3)


def _tie_batch(p, n, kind, seed=11):
    """A batch whose scores tie (one or two feasible moves repeated), or
    whose feasible moves are a scattered few among infeasible ones."""
    inc = O.OracleModel(p).eval_incremental(p.x0, p.moves[:4096])
    feas = np.flatnonzero((inc["flag"] != 0) & (inc["mean"] != 0.0))
    infeas = np.flatnonzero(inc["flag"] == 0)
    rng = np.random.default_rng(seed)
    if kind == "same":
        return np.repeat(p.moves[feas[:1]], n, axis=0)
    if kind == "two":
        pick = feas[:2][rng.integers(0, 2, n)]
        return p.moves[pick].copy()
    # "sparse": 20 feasible moves at random places among infeasible ones
    mv = p.moves[infeas[rng.integers(0, len(infeas), n)]].copy()
    at = rng.choice(n, 20, replace=False)
    mv[at] = p.moves[feas[:20]]
    return mv


@pytest.mark.parametrize("name,n,kind", [("plain_50k", 262_144, "same"), ("plain_50k", 262_144, "two"),
                                         ("plain_50k", 262_144, "sparse"), ("plain_4k", 20_000, "same"),
                                         ("plain_4k", 20_000, "sparse")])
@pytest.mark.parametrize("k", [1, 32])
def test_step_tied_scores_and_few_lists(name, n, kind, k):
    """The launch's last CTA selects the 32 best keys from the keys no smaller
    than the 32nd list head, or from every key when fewer than 32 CTA lists
    are non-empty, and falls back to a merge tree when too many keys qualify.
    Tied scores (keys differing only in the move index) drive the fallback,
    a few scattered feasible moves leave most CTA lists empty: both must give
    the separate calls' selection (ties by index) and the same apply."""
    p = W.config(name)
    mv = torch.as_tensor(_tie_batch(p, n, kind), device="cuda")
    a, b = _pair(p)
    for _ in range(2):
        ra = a.search_step(mv, k=k, apply=True)
        rb = _separate(b, mv, k, True)
        c = _compare(ra, rb, k)
        s, f = ra[0].cpu().numpy(), ra[1].cpu().numpy()
        ri, _ = O.topk(s.astype(np.float64), f, k)
        assert len(ri) == c and np.array_equal(ra[2].cpu().numpy()[:c], ri)
        assert a.last_apply() == b.last_apply()
    assert np.array_equal(a.schedule_get(), b.schedule_get())
    assert np.array_equal(a.npv()[0], b.npv()[0])
