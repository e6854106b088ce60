"""Uncertainty weights sigma(s,t) (Eq. 12) on the GPU vs the FP64 oracle.

The weighted model keeps the ore margins in its FP32 rows and a table of
weighted discount differences; the fast evaluator (S % 4 == 0, equal masses)
and the general one (any S, unequal masses, the compensated or generic
option) must both match the oracle's weighted deltas within the usual FP32
bound, the flags bit for bit; applies must keep the FP64 NPV equal to the
oracle's weighted NPV of the new schedule; the search step (one fused launch
in the weighted fast form) must match the separate calls bit for bit and keep
its running state equal to a rebuild.  With all weights 1 the NPV equals the
unweighted model's bit for bit.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import all_moves, assert_close_floor, tiny_problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2511_18296_b300  # noqa: F401


def _models(p, sigma, preds=None):
    import paper_2511_18296_b300 as mm
    m = mm.Model.from_problem(p, preds=preds, sigma=sigma)
    om = O.OracleModel(p, preds=preds, sigma=sigma)
    assert m.schedule_set(p.x0) == om.feasible(p.x0)
    return m, om


def _eval(m, moves, kahan=False, generic=False):
    mv = torch.as_tensor(np.ascontiguousarray(moves, np.int32), device="cuda")
    score, feas, mean, delta = m.eval_deltas(mv, kahan=kahan, generic=generic)
    torch.cuda.synchronize()
    return dict(score=score.cpu().numpy(), flag=feas.cpu().numpy(), mean=mean.cpu().numpy(),
                delta=delta.cpu().numpy())


def _check(g, om, x, moves, what, rows=None):
    ref = om.eval_bruteforce(x, moves) if rows is None else om.eval_incremental(x, moves, want_delta=True)
    inc = om.eval_incremental(x, moves, want_floor_s=True)
    assert np.array_equal(g["flag"], ref["flag"]), f"{what}: flags differ"
    assert_close_floor(g["score"], ref["score"], inc["floor"], what=f"{what} score")
    assert_close_floor(g["mean"], ref["mean"], inc["floor"], what=f"{what} mean")
    assert_close_floor(g["delta"], ref["delta"], inc["floor_s"], what=f"{what} delta")


def _margin_rows(p, om):
    m = p.mass.astype(np.float64)[:, None]
    margin = m * ((om.grade * p.price) * p.recovery - p.proc_cost)
    return np.where(om.ore == 1, margin, 0.0).astype(np.float32)


@pytest.mark.parametrize("S", [4, 8, 3, 13])
def test_tiny_models_every_move(S):
    """S = 4, 8: the fast form; S = 3, 13: the general kernel."""
    for seed, (nx, ny, nz, T, cap) in enumerate([(3, 3, 3, 3, 10), (4, 3, 2, 4, 7)]):
        p = tiny_problem(nx=nx, ny=ny, nz=nz, S=S, T=T, cap_blocks=cap, seed=seed + 10 * S)
        sigma = W.uncertainty_weights(T, S, seed=seed)
        m, om = _models(p, sigma)
        assert np.array_equal(m.values(), _margin_rows(p, om))
        mv = np.concatenate([all_moves(p.B, p.T), [[p.B, -1], [0, -(p.T + 2)]]]).astype(np.int32)
        _check(_eval(m, mv), om, p.x0, mv, f"S={S} seed={seed}")


def test_unequal_masses_and_csr():
    p = tiny_problem(nx=6, ny=1, nz=1, S=8, T=3, cap_blocks=3, seed=3, x0=[0, 0, 1, 1, 1, 2],
                     mass=[9000, 10000, 11000, 10000, 12000, 8000])
    ptr = np.array([0, 0, 0, 2, 3, 4, 6], np.int32)
    idx = np.array([0, 1, 2, 1, 4, 3], np.int32)
    sigma = W.uncertainty_weights(p.T, p.S, seed=5)
    m, om = _models(p, sigma, preds=(ptr, idx))
    mv = all_moves(p.B, p.T)
    _check(_eval(m, mv), om, p.x0, mv, "unequal masses")


@pytest.mark.parametrize("kahan,generic", [(False, False), (True, False), (False, True)])
def test_4k_every_move(kahan, generic):
    p = W.config("plain_4k")
    m, om = _models(p, W.uncertainty_weights(p.T, p.S))
    _check(_eval(m, p.moves, kahan=kahan, generic=generic), om, p.x0, p.moves, f"4k kahan={kahan} generic={generic}")


def test_50k_sample():
    p = W.config("plain_50k")
    m, om = _models(p, W.uncertainty_weights(p.T, p.S))
    g = _eval(m, p.moves)
    sel = np.sort(np.random.default_rng(12).choice(p.moves.shape[0], 1500, replace=False))
    gs = {k: v[sel] for k, v in g.items()}
    _check(gs, om, p.x0, p.moves[sel], "50k sample", rows=True)
    npv, mean, sd = m.npv()
    np.testing.assert_allclose(npv, om.npv(p.x0), rtol=1e-12)


def test_unit_weights_leave_the_npv_unchanged():
    import paper_2511_18296_b300 as mm
    p = W.config("plain_4k", n_moves=0)
    a = mm.Model.from_problem(p)
    b = mm.Model.from_problem(p, sigma=np.ones((p.T, p.S)))
    a.schedule_set(p.x0)
    b.schedule_set(p.x0)
    assert np.array_equal(a.npv()[0], b.npv()[0])


def test_applies_track_the_weighted_npv():
    p = W.config("plain_4k")
    sigma = W.uncertainty_weights(p.T, p.S, seed=9)
    m, om = _models(p, sigma)
    x = p.x0.copy()
    inc = om.eval_incremental(x, p.moves)
    order = np.argsort(-np.where(inc["flag"] == 1, inc["score"], -np.inf))
    applied = 0
    for j in order[:200]:
        b1, arg = (int(v) for v in p.moves[j])
        if om.apply(x, (b1, arg)) != 0:
            continue
        m.apply_move((b1, arg))
        applied += 1
    assert applied > 50
    assert np.array_equal(m.schedule_get(), x)
    np.testing.assert_allclose(m.npv()[0], om.npv(x), rtol=1e-10, atol=1e-3)


def test_search_step_matches_separate_calls():
    p = W.config("plain_4k")
    sigma = W.uncertainty_weights(p.T, p.S, seed=2)
    (a, om), (b, _) = _models(p, sigma), _models(p, sigma)
    mv = torch.as_tensor(p.moves, device="cuda")
    x = p.x0.copy()
    for _ in range(8):
        s, f, ia, ta, ca = a.search_step(mv, k=16, apply=True)
        sb, fb, _ = b.eval_moves(mv, want_mean=False)
        ib, tb, cb = b.topk(sb, fb, 16)
        b.apply_best(mv, ib, cb)
        torch.cuda.synchronize()
        assert np.array_equal(s.cpu().numpy().view(np.uint32), sb.cpu().numpy().view(np.uint32))
        c = int(ca.cpu()[0])
        assert c == int(cb.cpu()[0]) and np.array_equal(ia.cpu().numpy()[:c], ib.cpu().numpy()[:c])
        if c:
            j = int(ia.cpu()[0])
            assert om.apply(x, tuple(int(v) for v in p.moves[j])) == 0
        assert a.last_apply() == b.last_apply()
    assert np.array_equal(a.schedule_get(), x) and np.array_equal(b.schedule_get(), x)
    np.testing.assert_allclose(a.npv()[0], om.npv(x), rtol=1e-10, atol=1e-3)


def test_weighted_model_refused_by_relaxed_and_batch():
    import paper_2511_18296_b300 as mm
    p = W.config("plain_4k")
    m, _ = _models(p, W.uncertainty_weights(p.T, p.S))
    x = torch.as_tensor(W.relaxed_x(p.B, p.T, 2), device="cuda")
    with pytest.raises(mm.MMError):
        m.relaxed_forward(x)
    mv = torch.as_tensor(p.moves, device="cuda")
    with pytest.raises(mm.MMError):
        mm.Batch([(m, mv)], k=8)


def test_bad_weights_rejected():
    import paper_2511_18296_b300 as mm
    p = tiny_problem(S=4, T=3)
    for bad in (np.full((3, 4), np.nan), np.full((3, 4), -1.0)):
        with pytest.raises(mm.MMError):
            mm.Model.from_problem(p, sigma=bad)


@pytest.mark.parametrize("name,steps", [("plain_4k", 40), ("plain_50k", 15)])
def test_fused_weighted_step_state_matches_rebuild(name, steps):
    """The fused step in its weighted form (S % 4 == 0, equal masses): after
    every step the running FP64 state equals a fresh weighted model rebuilt
    from the same schedule (the in-launch apply uses the weighted margin)."""
    import paper_2511_18296_b300 as mm
    p = W.config(name)
    sigma = W.uncertainty_weights(p.T, p.S, seed=3)
    a = mm.Model.from_problem(p, sigma=sigma)
    fresh = mm.Model.from_problem(p, sigma=sigma)
    a.schedule_set(p.x0)
    mv = torch.as_tensor(p.moves, device="cuda")
    for _ in range(steps):
        a.search_step(mv, k=8, apply=True)
        assert a.last_apply()[0] == 1
        fresh.schedule_set(a.schedule_get())
        ma, oa = a.tonnage()
        mf, of = fresh.tonnage()
        assert np.array_equal(ma, mf) and np.array_equal(oa, of)
        np.testing.assert_allclose(a.metal(), fresh.metal(), rtol=1e-12, atol=1e-6)
        np.testing.assert_allclose(a.npv()[0], fresh.npv()[0], rtol=1e-12, atol=1e-3)
