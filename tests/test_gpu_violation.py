"""mm_eval_violation against the FP64 oracle's brute force, bit for bit.

Capacity excess (tonnes) and precedence excess (periods) are exact integers,
so the GPU must reproduce the oracle exactly: every move of tiny models (grid
and explicit-DAG precedence, adjacent swaps, unmined targets, no-ops, bad
moves, an over-full base schedule), all 4,096 moves of the 4k workload and a
sample of the 50k workload; both magnitudes are zero exactly when the GPU's
own feasibility flag is 1.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import all_moves, tiny_problem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _check(p, moves, preds=None, sample=None):
    import paper_2511_18296_b300 as mm
    m = mm.Model.from_problem(p, preds=preds)
    m.schedule_set(p.x0)
    mv = torch.as_tensor(np.ascontiguousarray(moves, np.int32), device="cuda")
    ce, pe = m.eval_violation(mv)
    _, f, _ = m.eval_moves(mv, want_mean=False)
    torch.cuda.synchronize()
    ce, pe, f = ce.cpu().numpy(), pe.cpu().numpy(), f.cpu().numpy().astype(bool)
    sel = np.arange(len(moves)) if sample is None else sample
    rce, rpe = O.OracleModel(p, preds=preds).violation(p.x0, moves[sel])
    assert np.array_equal(ce[sel], rce), "capacity excess differs from the oracle"
    assert np.array_equal(pe[sel], rpe), "precedence excess differs from the oracle"
    good = ce >= 0
    assert np.array_equal(((ce == 0) & (pe == 0))[good], f[good])
    return m


def test_tiny_models_every_move():
    for seed, (nx, ny, nz, T, cap) in enumerate([(3, 3, 3, 3, 10), (4, 3, 2, 4, 7), (3, 2, 3, 2, 12)]):
        p = tiny_problem(nx=nx, ny=ny, nz=nz, T=T, cap_blocks=cap, seed=seed)
        mv = np.concatenate([all_moves(p.B, p.T), [[p.B, -1], [0, -(p.T + 2)], [0, p.B], [-1, 0]]]).astype(np.int32)
        _check(p, mv)
        p.cap = np.full(T, (cap - 2) * 10_000, np.uint64)  # over-full base schedule
        _check(p, mv)


def test_explicit_dag_every_move():
    # a hand-made DAG in CSR form: 0 -> 2, 1 -> 2, 2 -> 3, 1 -> 4, 4 -> 5, 3 -> 5
    p = tiny_problem(nx=6, ny=1, nz=1, T=3, cap_blocks=3, seed=3, x0=[0, 0, 1, 1, 1, 2])
    ptr = np.array([0, 0, 0, 2, 3, 4, 6], np.int32)
    idx = np.array([0, 1, 2, 1, 4, 3], np.int32)
    _check(p, all_moves(p.B, p.T), preds=(ptr, idx))


def test_4k_every_move():
    p = W.config("plain_4k")
    _check(p, p.moves)


def test_50k_sample():
    p = W.config("plain_50k")
    sample = np.sort(np.random.default_rng(11).choice(p.moves.shape[0], 1500, replace=False))
    m = _check(p, p.moves, sample=sample)
    with pytest.raises(Exception):
        m.eval_violation(torch.zeros((0, 2), dtype=torch.int64, device="cuda"))


def test_period_limit_every_move():
    """T = 254 (the limit), blocks spread over the periods, one block of
    capacity per period so that many shifts overfill their target period."""
    B, T = 27, 254
    x0 = np.minimum(np.arange(B) * (T // B), T - 1).astype(np.uint8)
    p = tiny_problem(S=4, T=T, cap_blocks=1, seed=11, x0=x0)
    mv = np.concatenate([all_moves(p.B, p.T), [[0, -(p.T + 2)]]]).astype(np.int32)
    _check(p, mv)
