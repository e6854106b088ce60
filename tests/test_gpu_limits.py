"""Period counts past the period-pair table and up to the limit (T = 254).

Above 64 periods the model keeps no period-pair table, so the evaluator leaves
its compile-time-shaped fast form; at every such T it must still match the
FP64 oracle's brute force on every move of small models (flags bit for bit,
scores and means within the FP32 bound), with schedules spread over the high
periods so that large period indices reach the tables.  The fused step must
equal the separate calls bit for bit and keep its running state equal to a
rebuild; the weighted model (general kernel there) must match the weighted
oracle; T = 255 is refused.
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


def _spread_problem(T, S=8, seed=3):
    """27 blocks (3x3x3) placed one per period at spacing T // 27: feasible
    (periods grow with depth) and reaching far into the period range."""
    B = 27
    x0 = np.minimum(np.arange(B) * max(1, T // B), T - 1).astype(np.uint8)
    return tiny_problem(S=S, T=T, cap_blocks=2, target_blocks=1, seed=seed, x0=x0)


def _check(m, om, x, mv, what, kahan=False):
    s, f, mean = m.eval_moves(torch.as_tensor(mv, device="cuda"), kahan=kahan)
    torch.cuda.synchronize()
    ref = om.eval_bruteforce(x, mv)
    inc = om.eval_incremental(x, mv)
    assert np.array_equal(f.cpu().numpy(), ref["flag"]), f"{what}: flags differ"
    assert_close_floor(s.cpu().numpy(), ref["score"], inc["floor"], what=f"{what} score")
    assert_close_floor(mean.cpu().numpy(), ref["mean"], inc["floor"], what=f"{what} mean")


@pytest.mark.parametrize("T", [65, 128, 254])
def test_every_move_at_many_periods(T):
    import paper_2511_18296_b300 as mm
    p = _spread_problem(T)
    om = O.OracleModel(p)
    m = mm.Model.from_problem(p)
    assert m.schedule_set(p.x0) == om.feasible(p.x0)
    mv = all_moves(p.B, p.T)
    for kahan in (False, True):
        _check(m, om, p.x0, mv, f"T={T} kahan={kahan}", kahan=kahan)


@pytest.mark.parametrize("T", [65, 254])
def test_fused_step_at_many_periods(T):
    import paper_2511_18296_b300 as mm
    p = _spread_problem(T, S=16, seed=4)
    a = mm.Model.from_problem(p)
    b = mm.Model.from_problem(p)
    fresh = mm.Model.from_problem(p)
    a.schedule_set(p.x0)
    b.schedule_set(p.x0)
    mv = torch.as_tensor(all_moves(p.B, p.T), device="cuda")
    applied = 0
    for _ in range(12):
        s, f, ia, ta, ca = a.search_step(mv, k=8, apply=True)
        sb, fb, _ = b.eval_moves(mv, want_mean=False)
        ib, tb, cb = b.topk(sb, fb, 8)
        b.apply_best(mv, ib, cb)
        torch.cuda.synchronize()
        assert np.array_equal(s.cpu().numpy().view(np.uint32), sb.cpu().numpy().view(np.uint32))
        assert np.array_equal(f.cpu().numpy(), fb.cpu().numpy())
        c = int(ca.cpu()[0])
        assert c == int(cb.cpu()[0]) and np.array_equal(ia.cpu().numpy()[:c], ib.cpu().numpy()[:c])
        assert a.last_apply() == b.last_apply()
        applied += a.last_apply()[0]
        fresh.schedule_set(a.schedule_get())
        ma, oa = a.tonnage()
        mf, of = fresh.tonnage()
        assert np.array_equal(ma, mf) and np.array_equal(oa, of)
        np.testing.assert_allclose(a.npv()[0], fresh.npv()[0], rtol=1e-12, atol=1e-6)
    assert applied > 0
    assert np.array_equal(a.schedule_get(), b.schedule_get())


def test_weighted_at_many_periods():
    import paper_2511_18296_b300 as mm
    p = _spread_problem(100, S=8, seed=6)
    sigma = W.uncertainty_weights(p.T, p.S, seed=7)
    om = O.OracleModel(p, sigma=sigma)
    m = mm.Model.from_problem(p, sigma=sigma)
    m.schedule_set(p.x0)
    _check(m, om, p.x0, all_moves(p.B, p.T), "weighted T=100")
    np.testing.assert_allclose(m.npv()[0], om.npv(p.x0), rtol=1e-12)


def test_too_many_periods_refused():
    import paper_2511_18296_b300 as mm
    p = tiny_problem(S=4, T=255, x0=np.zeros(27, np.uint8))
    with pytest.raises(mm.MMError) as e:
        mm.Model.from_problem(p)
    assert e.value.status == 1
