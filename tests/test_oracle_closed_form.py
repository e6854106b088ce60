"""Closed forms for one scenario with a constant grade everywhere (oracle only).

With S = 1 and every block holding grade c, every block has the same value v and
the same ore bit, so per-period ore tonnage is (blocks in period) * m * ore.
A shift of one block from t to t' then changes the NPV by
    v (d_t' - d_t) - d_t [pen(O_t - dm) - pen(O_t)] - d_t' [pen(O_t' + dm) - pen(O_t')]
with dm = m if the grade is ore else 0, and any swap changes nothing.
The per-block value is written out from the economics (54 $ per g/t per
tonne of ore after recovery, 20 $/t processing, 2 $/t mining).
"""

import numpy as np
import pytest

import oracle as O
from helpers import all_moves, tiny_problem


def pen(o, q, a=2.0, e=4.0):
    return a * max(0, q - o) + e * max(0, o - q)


@pytest.mark.parametrize("c", [1.0, 0.2, 0.9])
def test_shift_closed_form_constant_grade(c):
    nx, ny, nz, T = 3, 2, 2, 4
    B = nx * ny * nz
    m = 10_000
    x0 = np.array([0, 0, 0, 0, 0, 0, 1, 1, 1, 2, 2, 3], np.uint8)  # top level first
    p = tiny_problem(nx, ny, nz, S=1, T=T, cap_blocks=7, target_blocks=2, grade=np.full((B, 1), c), x0=x0)
    om = O.OracleModel(p)
    ore = c * 60 * 0.9 > 20
    v = m * (54 * c - 22) if ore else -2 * m
    d = [1.1 ** -t for t in range(T)] + [0.0]
    count = np.bincount(x0, minlength=T + 1)
    q = 2 * m
    dm = m if ore else 0
    mv = all_moves(B, T)
    r = om.eval_incremental(x0, mv, want_delta=True)
    rb = om.eval_bruteforce(x0, mv)
    for i, (b, arg) in enumerate(mv):
        if arg >= 0:
            expect = 0.0
        else:
            t, tn = int(x0[b]), -arg - 1
            if t == tn:
                expect = 0.0
            else:
                expect = v * (d[tn] - d[t])
                if t < T:
                    o = count[t] * dm
                    expect -= d[t] * (pen(o - dm, q) - pen(o, q))
                if tn < T:
                    o = count[tn] * dm
                    expect -= d[tn] * (pen(o + dm, q) - pen(o, q))
        assert r["delta"][i, 0] == pytest.approx(expect, rel=1e-12, abs=1e-6), (b, arg)
        assert rb["delta"][i, 0] == pytest.approx(expect, rel=1e-12, abs=1e-6), (b, arg)
        assert r["std"][i] == 0.0          # S = 1
        assert r["score"][i] == pytest.approx(expect, rel=1e-12, abs=1e-6)


def test_npv_closed_form_constant_grade():
    """NPV of a schedule with n_t blocks of value v in period t, S = 1."""
    nx, ny, nz, T = 2, 2, 2, 3
    B = 8
    c = 1.0
    x0 = np.array([0, 0, 0, 1, 1, 1, 2, 3], np.uint8)
    p = tiny_problem(nx, ny, nz, S=1, T=T, cap_blocks=3, target_blocks=2, grade=np.full((B, 1), c), x0=x0)
    om = O.OracleModel(p)
    m = 10_000
    v = m * (54 * c - 22)
    n = [3, 3, 1]
    expect = sum(1.1 ** -t * (n[t] * v - pen(n[t] * m, 2 * m)) for t in range(T))
    assert om.npv(x0)[0] == pytest.approx(expect, rel=1e-13)
