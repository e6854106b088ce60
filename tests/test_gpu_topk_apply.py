"""Top-k and apply on the GPU vs the oracle (needs a B300)."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import assert_close_floor, certified_swaps, tiny_problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def mm():
    import paper_2511_18296_b300 as m
    return m


def model_for(p):
    m = mm().Model.from_problem(p)
    m.schedule_set(p.x0)
    return m


def gpu_topk(m, score, feas, k):
    s = torch.as_tensor(np.asarray(score, np.float32), device="cuda")
    f = torch.as_tensor(np.asarray(feas, np.uint8), device="cuda")
    idx, top, cnt = m.topk(s, f, k)
    torch.cuda.synchronize()
    c = int(cnt.cpu()[0])
    return idx.cpu().numpy()[:c], top.cpu().numpy()[:c]


@pytest.fixture(scope="module")
def small_model():
    return model_for(tiny_problem(3, 3, 2, S=2, T=2))


@pytest.mark.parametrize("n,k", [(1, 1), (100, 7), (5000, 256), (262_144, 32), (262_144, 1024), (70_001, 1000)])
def test_topk_given_scores_exact(small_model, n, k):
    rng = np.random.default_rng(n + k)
    s = rng.normal(size=n).astype(np.float32) * 1e4
    s[rng.integers(0, n, n // 10 + 1)] = np.float32(17.0)     # many exact ties
    s[rng.integers(0, n, 3)] = -0.0
    s[rng.integers(0, n, 3)] = 0.0
    f = (rng.random(n) < 0.3).astype(np.uint8)
    gi, gt = gpu_topk(small_model, s, f, k)
    ri, rt = O.topk(s.astype(np.float64), f, k)
    assert np.array_equal(gi, ri)
    assert np.array_equal(gt.astype(np.float64), rt)


def test_topk_concentrated_bin(small_model):
    """Almost every candidate in one histogram bin (equal scores): the exact
    radix select on the low bits must still return the lowest indices."""
    n = 200_000
    s = np.full(n, 123.5, np.float32)
    s[::7] = np.nextafter(np.float32(123.5), np.float32(1e9))
    f = np.ones(n, np.uint8)
    for k in (1, 64, 1024):
        gi, _ = gpu_topk(small_model, s, f, k)
        ri, _ = O.topk(s.astype(np.float64), f, k)
        assert np.array_equal(gi, ri)


def test_topk_edges(small_model):
    gi, _ = gpu_topk(small_model, np.ones(50, np.float32), np.zeros(50, np.uint8), 5)
    assert gi.size == 0                                         # all infeasible
    gi, _ = gpu_topk(small_model, np.arange(10, dtype=np.float32), np.ones(10, np.uint8), 64)
    assert gi.tolist() == list(range(9, -1, -1))                # k > feasible count
    s = np.array([np.nan, 1.0, -np.inf, 2.0], np.float32)
    gi, _ = gpu_topk(small_model, s, np.ones(4, np.uint8), 4)
    assert gi.tolist() == [3, 1, 2]                              # NaN excluded
    e = torch.zeros(0, device="cuda")
    idx, top, cnt = small_model.topk(e, torch.zeros(0, dtype=torch.uint8, device="cuda"), 3)
    assert int(cnt.cpu()[0]) == 0


def test_topk_of_eval_vs_fp64_oracle():
    """Top-k indices from the GPU's FP32 scores vs the FP64 oracle's: identical
    except for pairs the oracle itself separates by less than the tolerance."""
    p = W.config("plain_50k")
    om = O.OracleModel(p)
    m = model_for(p)
    mv = torch.as_tensor(p.moves, device="cuda")
    s, f, _ = m.eval_moves(mv)
    idx, top, cnt = m.topk(s, f, 256)
    torch.cuda.synchronize()
    gi = idx.cpu().numpy()[:int(cnt.cpu()[0])]
    inc = om.eval_incremental(p.x0, p.moves)
    ri, rt = O.topk(inc["score"], inc["flag"], 256)
    # a swap only inside a certified near-tie: the oracle's two scores within 1e-5
    certified_swaps(gi, ri, inc["score"], inc["floor"])
    # and exact against the oracle's top-k of the GPU's own scores
    gi2, _ = O.topk(s.cpu().numpy().astype(np.float64), f.cpu().numpy(), 256)
    assert np.array_equal(gi, gi2)


def test_apply_sequence_matches_oracle():
    p = W.config("plain_4k")
    om = O.OracleModel(p)
    m = model_for(p)
    x = p.x0.copy()
    mv = torch.as_tensor(p.moves, device="cuda")
    applied = 0
    for step in range(40):
        s, f, _ = m.eval_moves(mv)
        idx, top, cnt = m.topk(s, f, 4)
        torch.cuda.synchronize()
        c = int(cnt.cpu()[0])
        if c == 0:
            break
        best = p.moves[int(idx.cpu()[0])]
        ref = om.eval_incremental(x, best[None, :])
        assert ref["flag"][0] == 1
        mean, sd = m.apply_move(tuple(best))
        assert om.apply(x, best) == 0
        applied += 1
        ref_npv = om.npv(x)
        assert mean == pytest.approx(ref_npv.mean(), rel=1e-12)
        assert sd == pytest.approx(ref_npv.std(), rel=1e-7, abs=1e-6)
        assert np.array_equal(m.schedule_get(), x)
        mined, oreT = m.tonnage()
        rm, ro = om.tonnage(x)
        assert np.array_equal(mined, rm) and np.array_equal(oreT, ro)
    assert applied >= 10
    # the evaluator sees the updated state: compare a fresh batch
    s, f, mean = m.eval_moves(mv)
    torch.cuda.synchronize()
    inc = om.eval_incremental(x, p.moves)
    assert np.array_equal(f.cpu().numpy(), inc["flag"])
    assert_close_floor(s.cpu().numpy(), inc["score"], inc["floor"], what="after applies")


def test_apply_infeasible_and_bad_change_nothing():
    p = W.config("plain_4k")
    om = O.OracleModel(p)
    m = model_for(p)
    inc = om.eval_incremental(p.x0, p.moves)
    bad_i = int(np.nonzero(inc["flag"] == 0)[0][0])
    with pytest.raises(mm().MMError) as e:
        m.apply_move(tuple(p.moves[bad_i]))
    assert e.value.status == 5
    with pytest.raises(mm().MMError) as e:
        m.apply_move((p.B + 5, -1))
    assert e.value.status == 6
    assert np.array_equal(m.schedule_get(), p.x0)
    npv, mean, _ = m.npv()
    np.testing.assert_allclose(npv, om.npv(p.x0), rtol=1e-12)


def test_apply_best_on_device():
    p = W.config("plain_4k")
    om = O.OracleModel(p)
    m = model_for(p)
    x = p.x0.copy()
    mv = torch.as_tensor(p.moves, device="cuda")
    for step in range(10):
        s, f, _ = m.eval_moves(mv)
        idx, top, cnt = m.topk(s, f, 1)
        best = p.moves[int(idx.cpu()[0])] if int(cnt.cpu()[0]) else None
        m.apply_best(mv, idx, cnt)
        applied, mean, sd = m.last_apply()
        if best is None:
            assert applied == 0
            break
        assert applied == 1 and om.apply(x, best) == 0
        assert mean == pytest.approx(om.npv(x).mean(), rel=1e-12)
    assert np.array_equal(m.schedule_get(), x)
