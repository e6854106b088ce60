"""Small shared test helpers (test-only; no arithmetic of the method here)."""

import json
import os

import numpy as np

from workloads import Problem, random_moves

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def problem_from_dict(d, moves=None, name="golden"):
    return Problem(
        name=name, nx=d["nx"], ny=d["ny"], nz=d["nz"], S=d["S"], T=d["T"],
        mass=np.asarray(d["mass"], np.uint32),
        grade=np.asarray(d["grade"], np.float64).reshape(-1, d["S"]),
        cap=np.asarray(d["cap"], np.uint64), target=np.asarray(d["target"], np.uint64),
        x0=np.asarray(d["x0"], np.uint8),
        moves=np.asarray(moves if moves is not None else np.zeros((0, 2)), np.int32).reshape(-1, 2),
        price=d["price"], recovery=d["recovery"], mining_cost=d["mining_cost"], proc_cost=d["proc_cost"],
        shortfall_pen=d["shortfall_pen"], excess_pen=d["excess_pen"], discount_rate=d["discount_rate"],
        lam=d["lam"])


def tiny_problem(nx=3, ny=3, nz=3, S=3, T=3, cap_blocks=None, target_blocks=4, seed=5, grade=None,
                 mass=None, x0=None, lam=0.5, cv=0.8, **kw):
    """A small random instance: grades lognormal iid per (block, scenario)."""
    B = nx * ny * nz
    rng = np.random.default_rng(seed)
    if grade is None:
        grade = rng.lognormal(-0.25, 0.7, size=(B, S))
    if mass is None:
        mass = np.full(B, 10_000, np.uint32)
    if cap_blocks is None:
        cap_blocks = -(-B // T) + 1
    cap = np.full(T, cap_blocks * 10_000, np.uint64)
    target = np.full(T, target_blocks * 10_000, np.uint64)
    if x0 is None:
        x0 = np.minimum(np.arange(B) // cap_blocks, T).astype(np.uint8)
    p = Problem(name="tiny", nx=nx, ny=ny, nz=nz, S=S, T=T, mass=np.asarray(mass, np.uint32),
                grade=np.asarray(grade, np.float64).reshape(B, S), cap=cap, target=target,
                x0=np.asarray(x0, np.uint8), moves=np.zeros((0, 2), np.int32), lam=lam, **kw)
    return p


def all_moves(B, T):
    """Every shift (b, t') with t' in 0..T and every ordered swap (b1, b2)."""
    mv = [(b, -(t + 1)) for b in range(B) for t in range(T + 1)]
    mv += [(b1, b2) for b1 in range(B) for b2 in range(B)]
    return np.asarray(mv, np.int32)


REL_TOL = 1e-5  # relative error bound on FP32 deltas and scores vs the FP64 oracle


def assert_close_floor(gpu, ref, floor, rel=REL_TOL, what=""):
    """|gpu - ref| <= rel * max(|ref|, floor), elementwise.

    ``floor`` is the oracle's per-move (or per-scenario) scale of the terms
    that were summed, so that cancellation near zero is judged against the size
    of what cancelled.  Where ref and floor are both 0 (a no-op move) the GPU
    value must be exactly 0; equal infinities (bad moves) match."""
    g = np.asarray(gpu, np.float64)
    r = np.asarray(ref, np.float64)
    f = np.broadcast_to(np.asarray(floor, np.float64), r.shape)
    both_inf = np.isinf(g) & np.isinf(r) & (np.sign(g) == np.sign(r))
    with np.errstate(invalid="ignore"):
        err = np.where(both_inf, 0.0, np.abs(g - r))
    tol = rel * np.maximum(np.abs(np.where(both_inf, 0.0, r)), f)
    bad = ~(err <= tol)
    if bad.any():
        k = np.argmax(np.where(bad, err / np.maximum(tol, 1e-300), 0))
        idx = np.unravel_index(k, r.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {bad.size} outside tolerance; worst at {idx}: "
                             f"gpu={g[idx]!r} ref={r[idx]!r} floor={f[idx]!r}")


def certified_swaps(gi, ri, ref_score, ref_floor, rel=REL_TOL):
    """Positions where the GPU's top-k indices gi differ from the FP64
    oracle's ri, each checked to be a certified near-tie: the oracle's own
    scores of the two moves within rel * max(|score|, floor) of each other (so
    FP32 rounding alone can order them either way).  Returns the count; raises
    if a swap is not certified or the lengths differ."""
    gi, ri = np.asarray(gi), np.asarray(ri)
    if gi.size != ri.size:
        raise AssertionError(f"top-k sizes differ: {gi.size} vs {ri.size}")
    bad = np.nonzero(gi != ri)[0]
    for j in bad:
        a, b = ref_score[gi[j]], ref_score[ri[j]]
        scale = max(abs(a), abs(b), ref_floor[gi[j]], ref_floor[ri[j]])
        if not abs(a - b) <= rel * scale:
            raise AssertionError(f"top-k position {j}: gpu move {gi[j]} vs oracle move {ri[j]}, oracle scores "
                                 f"{a!r} and {b!r} are not within {rel} of {scale!r}")
    return int(bad.size)
