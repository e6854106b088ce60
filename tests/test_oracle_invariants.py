"""Invariants of the move evaluator (oracle only)."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import tiny_problem


@pytest.fixture(scope="module")
def p4k():
    p = W.config("plain_4k", n_moves=512)
    return p, O.OracleModel(p)


def test_swap_identical_blocks_is_zero():
    B = 18
    g = np.random.default_rng(0).lognormal(size=(B, 3))
    g[5] = g[14]                      # blocks 5 and 14 identical, different periods
    p = tiny_problem(3, 3, 2, S=3, T=3, grade=g, cap_blocks=7)
    om = O.OracleModel(p)
    assert p.x0[5] != p.x0[14]
    r = om.eval_incremental(p.x0, np.array([[5, 14], [14, 5]], np.int32), want_delta=True)
    assert np.all(r["delta"] == 0.0)
    assert np.all(r["score"] == 0.0)
    rb = om.eval_bruteforce(p.x0, np.array([[5, 14]], np.int32))
    assert np.abs(rb["delta"]).max() < 1e-6


def test_move_then_inverse(p4k):
    p, om = p4k
    mv = p.moves[:64]
    r = om.eval_incremental(p.x0, mv, want_delta=True)
    for i, (b1, arg) in enumerate(mv):
        x1 = p.x0.copy()
        if arg >= 0:
            x1[b1], x1[arg] = p.x0[arg], p.x0[b1]
            inv = (b1, arg)
        else:
            x1[b1] = -arg - 1
            inv = (b1, -(int(p.x0[b1]) + 1))
        ri = om.eval_incremental(x1, np.array([inv], np.int32), want_delta=True)
        np.testing.assert_allclose(ri["delta"][0], -r["delta"][i], rtol=1e-12, atol=1e-6)


def test_lambda_zero_gives_mean(p4k):
    p, _ = p4k
    p0 = W.config("plain_4k", n_moves=512, lam=0.0)
    om0 = O.OracleModel(p0)
    r = om0.eval_incremental(p0.x0, p0.moves)
    assert np.array_equal(r["score"], r["mean"])


def test_shift_to_same_period_is_zero(p4k):
    p, om = p4k
    b = np.arange(0, 4000, 97, dtype=np.int32)
    mv = np.stack([b, -(p.x0[b].astype(np.int32) + 1)], axis=1)
    r = om.eval_incremental(p.x0, mv, want_delta=True)
    assert np.all(r["delta"] == 0.0) and np.all(r["flag"] == 1)
    rb = om.eval_bruteforce(p.x0, mv)
    assert np.all(rb["delta"] == 0.0)


def test_apply_matches_eval_and_conserves_tonnage(p4k):
    p, om = p4k
    r = om.eval_incremental(p.x0, p.moves, want_delta=True)
    feas = np.nonzero(r["flag"])[0][:20]
    x = p.x0.copy()
    base_mined = om.tonnage(x)[0].sum()
    for i in feas:
        x_before = x.copy()
        npv0 = om.npv(x_before)
        ri = om.eval_incremental(x_before, p.moves[i:i + 1], want_delta=True)
        st = om.apply(x, p.moves[i])
        if ri["flag"][0]:
            assert st == 0
            np.testing.assert_allclose(om.npv(x) - npv0, ri["delta"][0], rtol=1e-9, atol=1e-5)
            assert om.feasible(x)
        else:
            assert st == 1 and np.array_equal(x, x_before)
        assert om.tonnage(x)[0].sum() == base_mined   # no block leaves or enters the mine here


def test_ore_threshold_is_strict():
    """0.37037037037037035 is the double with (g*60)*0.9 == 20 exactly: the
    strict '>' of the ore rule makes it waste; the next double up is ore."""
    g = 0.37037037037037035
    assert (g * 60.0) * 0.9 == 20.0
    up = np.nextafter(g, np.inf)
    assert (up * 60.0) * 0.9 > 20.0
    p = tiny_problem(2, 1, 1, S=1, T=1, grade=np.array([[g], [up]]), cap_blocks=2)
    om = O.OracleModel(p)
    assert om.ore[:, 0].tolist() == [0, 1]
    assert om.value[0, 0] == -2.0 * 10_000
