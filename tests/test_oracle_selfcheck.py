"""Brute force (full NPV recompute per move) vs the independent incremental
evaluator, exhaustively on tiny models and on every move of the 4k workload."""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import all_moves, tiny_problem


@pytest.mark.parametrize("S", [1, 2, 3])
@pytest.mark.parametrize("T", [2, 3])
def test_exhaustive_tiny(S, T):
    p = tiny_problem(3, 3, 3, S=S, T=T, seed=10 * S + T, target_blocks=5)
    om = O.OracleModel(p)
    mv = all_moves(p.B, T)
    bf = om.eval_bruteforce(p.x0, mv)
    inc = om.eval_incremental(p.x0, mv, want_delta=True)
    scale = np.abs(bf["delta"]).max()
    assert np.abs(bf["delta"] - inc["delta"]).max() <= 1e-12 * scale + 1e-9
    assert np.array_equal(bf["flag"], inc["flag"])
    np.testing.assert_allclose(bf["score"], inc["score"], rtol=1e-12, atol=1e-9 * scale)


def test_nonuniform_mass():
    rng = np.random.default_rng(4)
    B = 18
    mass = rng.integers(5_000, 15_000, size=B).astype(np.uint32)
    x0 = W.greedy_schedule(mass, np.full(3, 70_000, np.uint64), 3)
    p = tiny_problem(3, 3, 2, S=4, T=3, mass=mass, x0=x0, cap_blocks=7, target_blocks=3)
    om = O.OracleModel(p)
    assert om.feasible(x0)
    mv = all_moves(B, 3)
    bf = om.eval_bruteforce(x0, mv)
    inc = om.eval_incremental(x0, mv, want_delta=True)
    assert np.abs(bf["delta"] - inc["delta"]).max() <= 1e-6
    assert np.array_equal(bf["flag"], inc["flag"])


def test_plain_4k_every_move():
    p = W.config("plain_4k")
    om = O.OracleModel(p)
    assert om.feasible(p.x0)
    bf = om.eval_bruteforce(p.x0, p.moves)
    inc = om.eval_incremental(p.x0, p.moves, want_delta=True)
    # brute force subtracts two NPVs of ~1e9: its own rounding is ~1e-7 absolute
    assert np.abs(bf["delta"] - inc["delta"]).max() < 1e-5
    assert np.array_equal(bf["flag"], inc["flag"])
    assert np.abs(bf["score"] - inc["score"]).max() < 1e-5
