"""Seeded input generator: determinism, shapes and the lognormal targets."""

import numpy as np

import workloads as W


def test_deterministic_and_shapes():
    a = W.config("plain_4k")
    b = W.config("plain_4k")
    assert np.array_equal(a.grade, b.grade) and np.array_equal(a.moves, b.moves)
    assert a.grade.shape == (4000, 16) and a.moves.shape == (4096, 2)
    assert a.x0.dtype == np.uint8 and np.bincount(a.x0).tolist() == [600] * 6 + [400]


def test_lognormal_targets():
    g = W.lognormal_grades(30, 30, 10, 32, mean=1.0, cv=0.8, rng_a=5.0, nugget=0.1, sill=1.0, seed=9)
    assert abs(g.mean() - 1.0) < 0.06
    assert abs(g.std() / g.mean() - 0.8) < 0.1
    y = np.log(g)
    assert abs(y.std() - np.sqrt(np.log1p(0.64))) < 0.05


def test_spatial_correlation_decays():
    y = W.gaussian_field(40, 40, 1, 8, rng_a=8.0, nugget=0.1, sill=1.0,
                         seed_seq=np.random.SeedSequence(3))[:, 0]
    def corr(lag):
        a, b = y[:, :, :-lag].ravel(), y[:, :, lag:].ravel()
        return np.corrcoef(a, b)[0, 1]
    c1, c4, c16 = corr(1), corr(4), corr(16)
    # exponential model, practical range 8: 0.9*exp(-3h/8) -> 0.62, 0.20, 0.002
    assert 0.45 < c1 < 0.8 and 0.05 < c4 < 0.4 and abs(c16) < 0.12
    assert c1 > c4 > c16


def test_moves_mix_and_validity():
    p = W.config("plain_4k")
    mv = p.moves
    shifts = mv[:, 1] < 0
    assert shifts.sum() == 2048
    tn = -mv[shifts, 1] - 1
    assert np.all(tn >= 0) and np.all(tn < p.T) and np.all(tn != p.x0[mv[shifts, 0]])
    sw = mv[~shifts]
    assert np.all(p.x0[sw[:, 0]] != p.x0[sw[:, 1]])
    # interleaved, not blocked
    assert 0.3 < shifts[:2048].mean() < 0.7
