"""Pins of the float64 relaxed-objective oracle (oracle.relaxed).

It is checked against things other than itself: the discrete FP64 C oracle
(a 0/1 schedule with a very sharp softplus must give the discrete NPV), a hand
evaluation of a one-block case, the closed-form gradient of the penalty-free
objective, central finite differences of its own formula and the invariants
of the risk term.
"""

import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle as O
import oracle.relaxed as R
import workloads as W
from helpers import tiny_problem


def one_hot(x0, T):
    x = np.zeros((x0.shape[0], T), np.float64)
    mined = x0 < T
    x[np.nonzero(mined)[0], x0[mined]] = 1.0
    return x


def test_sharp_softplus_reproduces_the_discrete_objective():
    """A 0/1 schedule with beta -> large: |sp_beta - max(0, .)| <= log 2 / beta
    per term, so the relaxed NPV_s equals the C oracle's discrete NPV_s (Eq. 14
    with the piecewise-linear penalty) to within (a + e) m_ref log 2 T / beta."""
    p = W.config("plain_4k")
    x = one_hot(p.x0, p.T)
    beta = 1e7
    parts = R.relaxed_parts(torch.tensor(x), torch.tensor(p.grade), p.mass.astype(np.float64),
                            p.target.astype(np.float64), p, beta=beta)
    ref = O.OracleModel(p).npv(p.x0)
    bound = (p.shortfall_pen + p.excess_pen) * R.M_REF * math.log(2.0) * p.T / beta
    got = parts["npv"].numpy()
    assert np.all(np.abs(got - ref) <= bound + 1e-10 * np.abs(ref)), np.max(np.abs(got - ref))
    # and the moved schedule of a tiny model (periods of every block differ)
    q = tiny_problem(3, 3, 3, S=5, T=3, seed=4, target_blocks=4)
    xq = one_hot(q.x0, q.T)
    pq = R.relaxed_parts(torch.tensor(xq), torch.tensor(q.grade), q.mass.astype(np.float64),
                         q.target.astype(np.float64), q, beta=beta)
    refq = O.OracleModel(q).npv(q.x0)
    assert np.allclose(pq["npv"].numpy(), refq, rtol=1e-10, atol=bound)


def test_one_block_by_hand():
    """B = S = T = 1, x = 0.5, g = 1 g/t (ore: 54 > 20), m = 10,000 t, Q = 20,000 t."""
    p = W.config("plain_4k", n_moves=0)
    x = torch.tensor([[0.5]], dtype=torch.float64, requires_grad=True)
    g = torch.tensor([[1.0]], dtype=torch.float64, requires_grad=True)
    parts = R.relaxed_parts(x, g, [10_000.0], [20_000.0], p)
    v = 10_000.0 * (1.0 * 60.0 * 0.9 - 20.0) - 10_000.0 * 2.0  # 320,000
    o = 5_000.0
    sp = lambda z: (max(10.0 * z, 0.0) + math.log1p(math.exp(-abs(10.0 * z)))) / 10.0
    pen = 2.0 * 1e4 * sp((20_000.0 - o) / 1e4) + 4.0 * 1e4 * sp((o - 20_000.0) / 1e4)
    npv = 0.5 * v - pen
    assert float(parts["J"].detach()) == pytest.approx(npv, rel=1e-15)
    gx, gg = torch.autograd.grad(parts["J"], (x, g))
    sig = lambda z: 1.0 / (1.0 + math.exp(-10.0 * z))
    dpen = -2.0 * sig((20_000.0 - o) / 1e4) + 4.0 * sig((o - 20_000.0) / 1e4)
    assert float(gx[0, 0]) == pytest.approx(v - dpen * 10_000.0, rel=1e-13)
    assert float(gg[0, 0]) == pytest.approx(0.5 * 10_000.0 * 60.0 * 0.9, rel=1e-15)


def test_penalty_free_gradient_closed_form():
    """a = e = 0 and lambda = 0: J = sum_{b,t} x[b,t] d_t mean_s v[b,s], so
    dJ/dx[b,t] = d_t mean_s v[b,s] and dJ/dg[b,s] = ore m p r sum_t d_t x[b,t] / S."""
    q = tiny_problem(4, 3, 2, S=6, T=4, seed=11)
    q = dataclasses.replace(q, shortfall_pen=0.0, excess_pen=0.0, lam=0.0)
    x = W.relaxed_x(q.B, q.T, 5).astype(np.float64)
    r = R.relaxed_grads(x, q.grade, q.mass.astype(np.float64), q.target.astype(np.float64), q)
    m = q.mass.astype(np.float64)[:, None]
    ore = (q.grade * q.price) * q.recovery > q.proc_cost
    v = np.where(ore, m * ((q.grade * q.price) * q.recovery - q.proc_cost) - m * q.mining_cost, -m * q.mining_cost)
    d = np.array([(1.1) ** (-t) for t in range(q.T)])
    np.testing.assert_allclose(r["gx"], d[None, :] * v.mean(axis=1)[:, None], rtol=1e-12)
    np.testing.assert_allclose(r["gg"], ore * m * q.price * q.recovery * (x @ d)[:, None] / q.S, rtol=1e-12)


def test_risk_term_invariants():
    q = tiny_problem(3, 3, 2, S=7, T=3, seed=2)
    x = torch.tensor(W.relaxed_x(q.B, q.T, 9), dtype=torch.float64)
    g = torch.tensor(q.grade)
    parts = R.relaxed_parts(x, g, q.mass.astype(np.float64), q.target.astype(np.float64), q)
    npv = parts["npv"].numpy()
    assert float(parts["std"]) == pytest.approx(np.std(npv), rel=1e-12)  # population std
    q0 = dataclasses.replace(q, lam=0.0)
    assert float(R.relaxed_objective(x, g, q.mass.astype(np.float64), q.target.astype(np.float64), q0)) == \
        pytest.approx(npv.mean(), rel=1e-14)
    q1 = tiny_problem(3, 3, 2, S=1, T=3, seed=2)
    p1 = R.relaxed_parts(x, torch.tensor(q1.grade), q1.mass.astype(np.float64), q1.target.astype(np.float64), q1)
    assert float(p1["std"]) == 0.0 and float(p1["J"]) == float(p1["npv"][0])


def test_autograd_matches_central_differences():
    """Central differences (step 1e-3) of the float64 formula on 64 x and 64 g
    coordinates; g coordinates are taken away from the ore threshold so that
    the step does not cross it."""
    q = tiny_problem(5, 4, 3, S=9, T=5, seed=21, target_blocks=6)
    x = W.relaxed_x(q.B, q.T, 2).astype(np.float64)
    r = R.relaxed_grads(x, q.grade, q.mass.astype(np.float64), q.target.astype(np.float64), q)
    mass, tgt = q.mass.astype(np.float64), q.target.astype(np.float64)
    xt, gt = torch.tensor(x), torch.tensor(q.grade)
    rng = np.random.default_rng(0)
    fx = lambda xx: R.relaxed_objective(xx, gt, mass, tgt, q)
    fg = lambda gg: R.relaxed_objective(xt, gg, mass, tgt, q)
    for _ in range(64):
        i, t = int(rng.integers(q.B)), int(rng.integers(q.T))
        fd = R.central_difference(fx, xt, (i, t))
        assert fd == pytest.approx(r["gx"][i, t], rel=1e-6, abs=1e-6 * np.abs(r["gx"]).max())
    margin = np.abs(q.grade * q.price * q.recovery - q.proc_cost) > 2e-3 * q.price * q.recovery
    cand = np.argwhere(margin)
    for j in rng.choice(len(cand), 64, replace=False):
        i, s = (int(v) for v in cand[j])
        fd = R.central_difference(fg, gt, (i, s))
        assert fd == pytest.approx(r["gg"][i, s], rel=1e-6, abs=1e-6 * np.abs(r["gg"]).max())


def test_incremental_differences_equal_full_reevaluation():
    """The linear-update central differences used at full size equal central
    differences by full re-evaluation of the formula."""
    q = tiny_problem(4, 4, 3, S=8, T=4, seed=31, target_blocks=5)
    x = W.relaxed_x(q.B, q.T, 3).astype(np.float64)
    mass, tgt = q.mass.astype(np.float64), q.target.astype(np.float64)
    xt, gt = torch.tensor(x), torch.tensor(q.grade)
    rng = np.random.default_rng(1)
    for _ in range(16):
        b, t = int(rng.integers(q.B)), int(rng.integers(q.T))
        full = R.central_difference(lambda xx: R.relaxed_objective(xx, gt, mass, tgt, q), xt, (b, t))
        assert R.central_difference_x(x, q.grade, mass, tgt, q, b, t) == pytest.approx(full, rel=1e-9, abs=1e-6)
    margin = np.argwhere(np.abs(q.grade * q.price * q.recovery - q.proc_cost) > 2e-3 * q.price * q.recovery)
    for j in rng.choice(len(margin), 16, replace=False):
        b, s_ = (int(v) for v in margin[j])
        full = R.central_difference(lambda gg: R.relaxed_objective(xt, gg, mass, tgt, q), gt, (b, s_))
        assert R.central_difference_g(x, q.grade, mass, tgt, q, b, s_) == pytest.approx(full, rel=1e-9, abs=1e-6)
