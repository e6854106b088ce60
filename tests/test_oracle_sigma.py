"""Uncertainty weights sigma(s,t) of Eq. 12 in the FP64 oracle.

Eq. 12 scales the processing margin (revenue - processing cost) of a block
mined in period t under scenario s by sigma(s,t); the mining cost (the
scenario-independent c_bt of Eq. 14) and the mill penalties stay unweighted.

Pinned by a hand-worked two-block, two-scenario column (every number derived
in the comments; the weights differ by period and scenario so that a
transposed index, a weighted mining cost or penalty, or a dropped discount
each change a value), by special cases (sigma = 1 reproduces the unweighted
objective bit for bit; sigma = 0 leaves only the mining cost and penalties,
checked against the tonnages), by structure (the NPV is affine in sigma and a
change of sigma(s0,t0) moves NPV_s0 alone, by d_t0 times the period's summed
ore margin), and by the two independently written move evaluators agreeing
with random weights on every move of tiny models.
"""

import numpy as np

import oracle as O
import workloads as W
from helpers import all_moves, tiny_problem

D1 = 1.0 / 1.1  # discount of period 1 at r = 10 %


def _column():
    # 1 x 1 x 2 column: block 0 on top of block 1 (arc 0 -> 1), 10 t each;
    # S = 2, T = 2, capacity 20 t and mill target Q = 10 t per period.
    # Grades: block 0 (1 g/t, 0), block 1 (0, 1 g/t).  With p*rec = 54 $/g,
    # pc = 20 $/t, mc = 2 $/t: 1 g/t is ore with margin 10 (54 - 20) = 340,
    # 0 g/t is waste; a = 2 $/t short, e = 4 $/t over.
    p = tiny_problem(nx=1, ny=1, nz=2, S=2, T=2, cap_blocks=2, target_blocks=1, x0=[0, 1], mass=[10, 10],
                     grade=[[1.0, 0.0], [0.0, 1.0]])
    p.cap = np.full(2, 20, np.uint64)
    p.target = np.full(2, 10, np.uint64)
    sigma = np.array([[0.5, 3.0],     # t = 0: sigma(0,0), sigma(1,0)
                      [2.0, 0.25]])   # t = 1: sigma(0,1), sigma(1,1)
    return p, sigma


def test_hand_worked_column():
    p, sigma = _column()
    om = O.OracleModel(p, sigma=sigma)
    # x = (0, 1).
    # s = 0: t0 holds block 0 (ore): 0.5*340 - 20 = 150, ore 10 t = Q (no penalty);
    #        t1 holds block 1 (waste): -20, ore 0 t: shortfall 2*10 = 20.
    #        NPV_0 = 150 + (-20 - 20) d1.
    # s = 1: t0: block 0 waste: -20, shortfall 20; t1: block 1 ore:
    #        0.25*340 - 20 = 65, ore 10 t = Q.  NPV_1 = -40 + 65 d1.
    npv = om.npv(p.x0)
    np.testing.assert_allclose(npv, [150 - 40 * D1, -40 + 65 * D1], rtol=1e-14)
    moves = np.array([
        (1, -1),  # shift block 1 to period 0: x' = (0, 0)
        (0, 1),   # swap blocks 0 and 1: x' = (1, 0) (breaks the arc 0 -> 1)
    ], np.int32)
    # shift: s = 0: t0 = 150 - 20 = 130 (ore 10 t), t1 empty: shortfall 20.
    #               NPV' = 130 - 20 d1, delta = -20 + 20 d1.
    #        s = 1: t0 = -20 + (3*340 - 20) = 980 (ore 10 t), t1 empty: -20 d1.
    #               delta = 980 - 20 d1 - (-40 + 65 d1) = 1020 - 85 d1.
    # swap:  s = 0: t0 block 1 waste: -20 - 20; t1 block 0 ore: (2*340 - 20) d1 = 660 d1.
    #               delta = -40 + 660 d1 - (150 - 40 d1) = -190 + 700 d1.
    #        s = 1: t0 block 1 ore: 3*340 - 20 = 1000; t1 block 0 waste: (-20 - 20) d1.
    #               delta = 1000 - 40 d1 - (-40 + 65 d1) = 1040 - 105 d1.
    want = np.array([[-20 + 20 * D1, 1020 - 85 * D1], [-190 + 700 * D1, 1040 - 105 * D1]])
    bf = om.eval_bruteforce(p.x0, moves)
    inc = om.eval_incremental(p.x0, moves, want_delta=True)
    np.testing.assert_allclose(bf["delta"], want, rtol=1e-13)
    np.testing.assert_allclose(inc["delta"], want, rtol=1e-13)
    assert bf["flag"].tolist() == [1, 0] and inc["flag"].tolist() == [1, 0]


def _models():
    for seed, (nx, ny, nz, S, T, cap) in enumerate([(3, 3, 3, 4, 3, 10), (4, 3, 2, 5, 4, 7), (3, 2, 3, 3, 2, 12)]):
        p = tiny_problem(nx=nx, ny=ny, nz=nz, S=S, T=T, cap_blocks=cap, seed=seed)
        yield p, W.uncertainty_weights(T, S, seed=seed + 20)


def test_unit_weights_reproduce_unweighted_objective():
    for p, _ in _models():
        ones = np.ones((p.T, p.S))
        a, b = O.OracleModel(p), O.OracleModel(p, sigma=ones)
        assert np.array_equal(a.npv(p.x0), b.npv(p.x0))  # 1.0 * margin - m mc == value, bit for bit
        mv = all_moves(p.B, p.T)
        assert np.array_equal(a.eval_bruteforce(p.x0, mv)["delta"], b.eval_bruteforce(p.x0, mv)["delta"])


def test_zero_weights_leave_mining_cost_and_penalties():
    for p, _ in _models():
        om = O.OracleModel(p, sigma=np.zeros((p.T, p.S)))
        mined, oreT = om.tonnage(p.x0)
        d = (1.0 + p.discount_rate) ** -np.arange(p.T)
        Q = p.target.astype(np.float64)[:, None]
        o = oreT.astype(np.float64)
        pen = p.shortfall_pen * np.maximum(Q - o, 0) + p.excess_pen * np.maximum(o - Q, 0)
        want = -(d[:, None] * (p.mining_cost * mined.astype(np.float64)[:, None] + pen)).sum(0)
        np.testing.assert_allclose(om.npv(p.x0), want, rtol=1e-12)


def test_affine_and_local_in_the_weights():
    rng = np.random.default_rng(7)
    for p, sigma in _models():
        def npv(sg):
            return O.OracleModel(p, sigma=sg).npv(p.x0)
        n0 = npv(np.zeros_like(sigma))
        s2 = rng.uniform(0.1, 2.0, sigma.shape)
        lhs = npv(sigma + s2) - n0
        rhs = (npv(sigma) - n0) + (npv(s2) - n0)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-6)
        # one weight changed: only its scenario moves, by d_t0 * delta * (summed
        # ore margin of the period), the margin being value + m mc of the
        # unweighted classification
        plain = O.OracleModel(p)
        d = (1.0 + p.discount_rate) ** -np.arange(p.T)
        for t0, s0 in [(0, 0), (p.T - 1, p.S - 1), (p.T // 2, 1)]:
            bumped = sigma.copy()
            bumped[t0, s0] += 0.5
            diff = npv(bumped) - npv(sigma)
            others = np.delete(diff, s0)
            assert np.all(others == 0.0)
            in_t0 = p.x0 == t0
            margin = (plain.value[in_t0, s0] + p.mass[in_t0] * p.mining_cost)[plain.ore[in_t0, s0] == 1].sum()
            np.testing.assert_allclose(diff[s0], 0.5 * d[t0] * margin, rtol=1e-9, atol=1e-6)
            assert diff[s0] >= 0.0  # ore margins are positive by the classification rule


def test_bruteforce_matches_incremental_every_move():
    for p, sigma in _models():
        om = O.OracleModel(p, sigma=sigma)
        mv = all_moves(p.B, p.T)
        bf = om.eval_bruteforce(p.x0, mv)
        inc = om.eval_incremental(p.x0, mv, want_delta=True, want_floor_s=True)
        tol = 1e-9 * np.maximum(np.abs(bf["delta"]), inc["floor_s"])
        assert np.all(np.abs(inc["delta"] - bf["delta"]) <= tol)
        assert np.array_equal(bf["flag"], inc["flag"])


def test_inverse_move_negates_delta():
    p, sigma = next(_models())
    om = O.OracleModel(p, sigma=sigma)
    rng = np.random.default_rng(3)
    for _ in range(40):
        b = int(rng.integers(p.B))
        t = int(rng.integers(p.T))
        x1 = p.x0.copy()
        x1[b] = t
        fwd = om.eval_bruteforce(p.x0, np.array([(b, -(t + 1))], np.int32))["delta"][0]
        back = om.eval_bruteforce(x1, np.array([(b, -(int(p.x0[b]) + 1))], np.int32))["delta"][0]
        np.testing.assert_allclose(fwd, -back, rtol=1e-12, atol=1e-6)
