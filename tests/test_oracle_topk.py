"""Oracle top-k vs Python's sorted() on (-score, index)."""

import numpy as np
import pytest

import oracle as O


def py_topk(score, flag, k):
    keys = sorted((-s, i) for i, (s, f) in enumerate(zip(score, flag)) if f)
    return [i for _, i in keys[:k]]


@pytest.mark.parametrize("k", [1, 5, 32, 300])
def test_random_with_ties(k):
    rng = np.random.default_rng(k)
    n = 257
    s = rng.integers(-5, 5, size=n).astype(np.float64)     # many exact ties
    s[rng.integers(0, n, 10)] = -0.0
    f = (rng.random(n) < 0.7).astype(np.uint8)
    idx, top = O.topk(s, f, k)
    assert idx.tolist() == py_topk(s, f, k)
    assert np.array_equal(top, s[idx])


def test_all_infeasible_and_empty():
    idx, _ = O.topk(np.ones(10), np.zeros(10, np.uint8), 4)
    assert idx.size == 0
    idx, _ = O.topk(np.ones(0), np.zeros(0, np.uint8), 4)
    assert idx.size == 0


def test_signed_zero_ties_by_index():
    s = np.array([-0.0, 0.0, -0.0, 0.0])
    idx, _ = O.topk(s, np.ones(4, np.uint8), 4)
    assert idx.tolist() == [0, 1, 2, 3]
