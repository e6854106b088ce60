"""Violation magnitudes (epsilon-relaxed fitness, Algorithm 2) in the FP64 oracle.

Pinned by a hand-worked column of three blocks (every number below is derived
in the comments from the definitions), by the invariant that both magnitudes
are zero exactly when the move's local feasibility flag is 1 (checked against
the independently written flag of the incremental evaluator over every move
of several tiny models and of the 4k workload), and by scaling: doubling every
block mass and capacity doubles the capacity excess and leaves the precedence
excess unchanged.
"""

import numpy as np

import oracle as O
import workloads as W
from helpers import all_moves, tiny_problem


def _column():
    # 1 x 1 x 3 column: block 0 on top, block 1 below it, block 2 at the bottom;
    # arcs 0 -> 1 and 1 -> 2.  T = 3, 10 t blocks, capacity one block (10 t)
    # per period, schedule x = (0, 1, 2).
    return tiny_problem(nx=1, ny=1, nz=3, S=2, T=3, cap_blocks=1, target_blocks=1, x0=[0, 1, 2],
                        mass=[10, 10, 10])


def test_hand_worked_column():
    p = _column()
    p.cap = np.full(3, 10, np.uint64)
    om = O.OracleModel(p)
    moves = np.array([
        (2, -1),   # block 2 -> period 0: x' = (0,1,0); period 0 holds 20 t (+10); pred 1 in period 1 > 0 (+1)
        (0, -3),   # block 0 -> period 2: x' = (2,1,2); period 2 holds 20 t (+10); succ 1 in period 1 < 2 (+1)
        (0, 2),    # swap 0 and 2: x' = (2,1,0); capacities fine; block 0: succ at 1 < 2 (+1); block 2: pred at 1 > 0 (+1)
        (0, 1),    # swap 0 and 1 (arc 0 -> 1): x' = (1,0,2); block 0: succ at 0 < 1 (+1); block 1: pred at 1 > 0 (+1)
        (1, -4),   # block 1 -> unmined (T = 3): x' = (0,3,2); period 1 empties; succ 2 at 2 < 3 (+1)
        (1, -2),   # block 1 -> its own period: nothing changes, nothing violated
        (1, 1),    # block 1 swapped with itself: nothing changes
        (5, -1),   # bad block id
        (0, -5),   # bad period (T + 1)
    ], np.int32)
    ce, pe = om.violation(p.x0, moves)
    assert ce.tolist() == [10, 10, 0, 0, 0, 0, 0, -1, -1]
    assert pe.tolist() == [1, 1, 2, 2, 1, 0, 0, -1, -1]


def _zero_iff_flag(p):
    om = O.OracleModel(p)
    moves = all_moves(p.B, p.T)
    ce, pe = om.violation(p.x0, moves)
    flag = om.eval_incremental(p.x0, moves)["flag"].astype(bool)
    assert np.all(ce >= 0) and np.all(pe >= 0)
    assert np.array_equal((ce == 0) & (pe == 0), flag)
    return ce, pe


def test_zero_exactly_when_feasible_tiny_models():
    for seed, (nx, ny, nz, T, cap) in enumerate([(3, 3, 3, 3, 10), (4, 3, 2, 4, 7), (3, 2, 3, 2, 12)]):
        p = tiny_problem(nx=nx, ny=ny, nz=nz, T=T, cap_blocks=cap, seed=seed)
        _zero_iff_flag(p)
        # an over-full base schedule: capacity excess appears on no-op moves too
        p2 = tiny_problem(nx=nx, ny=ny, nz=nz, T=T, cap_blocks=cap, seed=seed)
        p2.cap = np.full(T, (cap - 2) * 10_000, np.uint64)
        ce, _ = _zero_iff_flag(p2)
        assert (ce > 0).any()


def test_zero_exactly_when_feasible_4k_workload():
    p = W.config("plain_4k")
    om = O.OracleModel(p)
    ce, pe = om.violation(p.x0, p.moves)
    flag = om.eval_incremental(p.x0, p.moves)["flag"].astype(bool)
    assert np.array_equal((ce == 0) & (pe == 0), flag)
    assert (pe > 0).any() and (ce > 0).any()


def test_capacity_excess_scales_with_mass():
    p = tiny_problem(nx=3, ny=3, nz=2, T=3, cap_blocks=5, seed=9)
    moves = all_moves(p.B, p.T)
    ce1, pe1 = O.OracleModel(p).violation(p.x0, moves)
    p.mass = p.mass * 2
    p.cap = p.cap * 2
    ce2, pe2 = O.OracleModel(p).violation(p.x0, moves)
    assert np.array_equal(ce2, 2 * ce1) and np.array_equal(pe2, pe1)
