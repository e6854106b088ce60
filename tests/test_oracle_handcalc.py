"""Oracle vs a hand-computed 4-block example (tests/golden/handcalc_2x1x2.json).

The paper prints no worked example for the evaluator; the fixture derives every
number by hand from Eq. 14-16 and the ore/waste reading of Eq. 18, so a dropped
penalty, a wrong discount exponent, a flipped precedence arc, a sample (instead
of population) std or a wrong ore threshold each changes at least one value.
"""

import numpy as np
import pytest

import oracle as O
from helpers import load_golden, problem_from_dict

G = load_golden("handcalc_2x1x2.json")


@pytest.fixture(scope="module")
def om():
    p = problem_from_dict(G["problem"], G["moves"])
    return O.OracleModel(p), p


def test_stencil_matches_fixture():
    ptr, idx = O.stencil_preds(2, 1, 2)
    got = {f"b{b}": sorted(idx[ptr[b]:ptr[b + 1]].tolist()) for b in range(4)}
    assert got == G["preds"]


def test_classify(om):
    m, _ = om
    assert m.ore.tolist() == G["ore"]
    np.testing.assert_allclose(m.value, np.asarray(G["value"]), rtol=1e-12)


def test_npv(om):
    m, p = om
    np.testing.assert_allclose(m.npv(p.x0), G["npv"], rtol=1e-12)
    assert m.feasible(p.x0)


@pytest.mark.parametrize("evaluator", ["bruteforce", "incremental"])
def test_moves(om, evaluator):
    m, p = om
    r = m.eval_bruteforce(p.x0, p.moves) if evaluator == "bruteforce" else \
        m.eval_incremental(p.x0, p.moves, want_delta=True)
    assert r["flag"].tolist() == G["flag"]
    for i, name in enumerate(G["move_names"]):
        if G["delta_x11"][i] is None:
            assert r["score"][i] == -np.inf, name
            continue
        np.testing.assert_allclose(r["delta"][i], np.asarray(G["delta_x11"][i]) / 11.0, rtol=1e-12, atol=1e-9,
                                   err_msg=name)
        np.testing.assert_allclose(r["mean"][i], G["mean_x11"][i] / 11.0, rtol=1e-12, atol=1e-9, err_msg=name)
        np.testing.assert_allclose(r["std"][i], G["std_x11"][i] / 11.0, rtol=1e-12, atol=1e-9, err_msg=name)
        np.testing.assert_allclose(r["score"][i], G["score_x11"][i] / 11.0, rtol=1e-12, atol=1e-9, err_msg=name)


def test_top2(om):
    m, p = om
    r = m.eval_bruteforce(p.x0, p.moves)
    idx, _ = O.topk(r["score"], r["flag"], 2)
    assert idx.tolist() == G["top2"]


def test_apply_then_npv(om):
    m, p = om
    x = p.x0.copy()
    assert m.apply(x, (3, -3)) == 0            # move E: feasible
    assert x.tolist() == [0, 0, 1, 2]
    np.testing.assert_allclose(m.npv(x), np.array([9330 - 6100, 8730 + 200]) / 11.0, rtol=1e-12)
    x2 = p.x0.copy()
    assert m.apply(x2, (3, -1)) == 1           # move A: over capacity, no change
    assert x2.tolist() == p.x0.tolist()
    assert m.apply(x2, (4, -1)) == 2           # bad block id
