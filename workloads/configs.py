"""Synthetic problem instances shaped like the paper's workloads.

Five workloads are defined, each a plain dict of parameters:

* ``plain_4k``   - 20x20x10 = 4,000 blocks, S=16, T=8, 4,096 moves (small enough
  for the brute-force oracle on every move);
* ``plain_50k``  - 50x50x20 = 50,000 blocks, S=100, T=20, 262,144 moves: the
  paper's scale (more than 50,000 blocks, 262,144 simultaneous candidates,
  Table 5);
* ``batched_64`` - 64 independent chains of cubic models with side 15..40,
  S in {16, 32, 64, 100}, log-uniform move batches 1,024..65,536;
* ``relaxed_50k`` - the 50k model with a fractional schedule x[b,t] drawn from
  Dirichlet(1) per block;
* ``stress_400k`` - 100x100x40 = 400,000 blocks, S=500, T=30, 1,048,576 moves.

Economics shared by all of them: 10,000 t blocks, price 60 $/g, recovery 0.9,
mining cost 2 $/t, processing cost 20 $/t, mill shortfall penalty 2 $/t and
excess penalty 4 $/t, discount rate 10 % per period, risk weight lambda 0.5.

Nothing here evaluates a schedule: no ore/waste test, no values, no penalties.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .grf import lognormal_grades

BLOCK_T = 10_000  # tonnes per block

ECON = dict(
    price=60.0,
    recovery=0.9,
    mining_cost=2.0,
    proc_cost=20.0,
    shortfall_pen=2.0,
    excess_pen=4.0,
    discount_rate=0.10,
    lam=0.5,
)

CONFIGS = {
    "plain_4k": dict(nx=20, ny=20, nz=10, S=16, mean=1.0, cv=0.8, rng_a=5.0, nugget=0.1, sill=1.0,
                     seed=0, T=8, cap_blocks=600, target_blocks=250, n_moves=4096, shift_frac=0.5),
    "plain_50k": dict(nx=50, ny=50, nz=20, S=100, mean=1.0, cv=0.8, rng_a=8.0, nugget=0.1, sill=1.0,
                      seed=1, T=20, cap_blocks=2800, target_blocks=1100, n_moves=262_144, shift_frac=0.5),
    "relaxed_50k": dict(nx=50, ny=50, nz=20, S=100, mean=1.0, cv=0.8, rng_a=8.0, nugget=0.1, sill=1.0,
                        seed=1, T=20, cap_blocks=2800, target_blocks=1100, n_moves=0, shift_frac=0.5,
                        x_seed=2),
    "stress_400k": dict(nx=100, ny=100, nz=40, S=500, mean=1.0, cv=1.0, rng_a=12.0, nugget=0.1, sill=1.0,
                        seed=3, T=30, cap_blocks=14_000, target_blocks=5_500, n_moves=1_048_576,
                        shift_frac=0.7, n_applies=1000),
}


@dataclass
class Problem:
    """One block model, its scenarios, economics, an initial schedule and moves.

    Layouts: ``grade`` float64 [B][S] (scenario fastest); ``mass`` uint32 [B];
    ``cap`` / ``target`` uint64 [T] tonnes; ``x0`` uint8 [B] (value T = unmined);
    ``moves`` int32 [n][2] = (b1, arg): arg >= 0 swaps b1 with block arg,
    arg < 0 shifts b1 to period -arg-1.
    """

    name: str
    nx: int
    ny: int
    nz: int
    S: int
    T: int
    mass: np.ndarray
    grade: np.ndarray
    cap: np.ndarray
    target: np.ndarray
    x0: np.ndarray
    moves: np.ndarray
    price: float = ECON["price"]
    recovery: float = ECON["recovery"]
    mining_cost: float = ECON["mining_cost"]
    proc_cost: float = ECON["proc_cost"]
    shortfall_pen: float = ECON["shortfall_pen"]
    excess_pen: float = ECON["excess_pen"]
    discount_rate: float = ECON["discount_rate"]
    lam: float = ECON["lam"]
    extra: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return self.nx * self.ny * self.nz


def greedy_schedule(mass: np.ndarray, cap: np.ndarray, T: int) -> np.ndarray:
    """Fill periods in raster order (b = x + nx*(y + ny*z), top level first).

    Each block goes to the current period while that period's mined tonnage
    stays within its capacity, else to the next period; blocks left over after
    the last period stay unmined (period value T).  Because predecessors sit on
    the level above, and so earlier in raster order, the result respects
    precedence.
    """
    B = mass.shape[0]
    x = np.full(B, T, dtype=np.uint8)
    t = 0
    used = 0
    for b in range(B):
        m = int(mass[b])
        while t < T and used + m > int(cap[t]):
            t += 1
            used = 0
        if t >= T:
            break
        x[b] = t
        used += m
    return x


def greedy_schedule_uniform(B: int, cap_blocks: int, T: int) -> np.ndarray:
    """Closed form of greedy_schedule for equal block masses: x_b = b // cap."""
    x = np.arange(B, dtype=np.int64) // cap_blocks
    x = np.minimum(x, T)
    return x.astype(np.uint8)


def random_moves(x: np.ndarray, T: int, n: int, shift_frac: float,
                 rng: np.random.Generator) -> np.ndarray:
    """n moves: round(shift_frac*n) shifts, the rest swaps, randomly interleaved.

    Shift: block uniform, new period uniform over the T-1 periods other than the
    block's current one (an unmined block draws from periods 0..T-2).  Swap: a uniform pair of blocks in different periods
    (redrawn until the periods differ).
    """
    B = x.shape[0]
    n_shift = int(round(shift_frac * n))
    n_swap = n - n_shift
    mv = np.empty((n, 2), dtype=np.int32)
    # shifts
    b = rng.integers(0, B, size=n_shift)
    cur = x[b].astype(np.int64)
    cur_c = np.minimum(cur, T - 1)
    r = rng.integers(0, T - 1, size=n_shift)
    tnew = np.where(r >= cur_c, r + 1, r)
    tnew = np.where(cur >= T, r, tnew)
    mv[:n_shift, 0] = b
    mv[:n_shift, 1] = -(tnew + 1)
    # swaps, redrawn until the two periods differ
    b1 = rng.integers(0, B, size=n_swap)
    b2 = rng.integers(0, B, size=n_swap)
    bad = x[b1] == x[b2]
    while bad.any():
        k = int(bad.sum())
        b1[bad] = rng.integers(0, B, size=k)
        b2[bad] = rng.integers(0, B, size=k)
        bad = x[b1] == x[b2]
    mv[n_shift:, 0] = b1
    mv[n_shift:, 1] = b2
    perm = rng.permutation(n)
    return np.ascontiguousarray(mv[perm])


def make_problem(name: str, nx: int, ny: int, nz: int, S: int, T: int, cap_blocks: int,
                 target_blocks: int, n_moves: int, shift_frac: float, seed: int,
                 mean: float = 1.0, cv: float = 0.8, rng_a: float = 5.0, nugget: float = 0.1,
                 sill: float = 1.0, grade: Optional[np.ndarray] = None,
                 mass: Optional[np.ndarray] = None, x0: Optional[np.ndarray] = None,
                 **econ) -> Problem:
    """Build one Problem.  ``grade``, ``mass`` and ``x0`` may be given directly
    (small hand-made cases); otherwise they come from the seeded generator."""
    B = nx * ny * nz
    if grade is None:
        grade = lognormal_grades(nx, ny, nz, S, mean, cv, rng_a, nugget, sill, seed)
    grade = np.ascontiguousarray(grade, dtype=np.float64).reshape(B, S)
    if mass is None:
        mass = np.full(B, BLOCK_T, dtype=np.uint32)
    mass = np.ascontiguousarray(mass, dtype=np.uint32)
    cap = np.full(T, cap_blocks * BLOCK_T, dtype=np.uint64)
    target = np.full(T, target_blocks * BLOCK_T, dtype=np.uint64)
    if x0 is None:
        if np.all(mass == BLOCK_T):
            x0 = greedy_schedule_uniform(B, cap_blocks, T)
        else:
            x0 = greedy_schedule(mass, cap, T)
    x0 = np.ascontiguousarray(x0, dtype=np.uint8)
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(2)[1])
    moves = random_moves(x0, T, n_moves, shift_frac, rng) if n_moves > 0 else np.zeros((0, 2), np.int32)
    e = dict(ECON)
    e.update(econ)
    return Problem(name=name, nx=nx, ny=ny, nz=nz, S=S, T=T, mass=mass, grade=grade, cap=cap,
                   target=target, x0=x0, moves=moves, **e)


def config(name: str, n_moves: Optional[int] = None, **over) -> Problem:
    """Problem for one named workload (optionally with fewer moves)."""
    p = dict(CONFIGS[name])
    p.update(over)
    if n_moves is not None:
        p["n_moves"] = n_moves
    extra = {k: p.pop(k) for k in ("x_seed", "n_applies") if k in p}
    prob = make_problem(name, **p)
    prob.extra.update(extra)
    return prob


def batched_chain_specs(n_chains: int = 64, base_seed: int = 100) -> list:
    """Per-chain parameters of the batched multi-chain workload.

    Chain c uses seed base_seed + c.  Cube side uniform in 15..40, S uniform in
    {16, 32, 64, 100}, T = 20, move-batch size log-uniform in 1,024..65,536,
    capacity ceil(1.12 * B / T) blocks and mill target round(0.393 * capacity)
    blocks (the capacity and target ratios of the 50k workload), half shifts.
    """
    specs = []
    for c in range(n_chains):
        seed = base_seed + c
        rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
        side = int(rng.integers(15, 41))
        S = int(rng.choice([16, 32, 64, 100]))
        n = int(round(math.exp(rng.uniform(math.log(1024), math.log(65536)))))
        B = side ** 3
        T = 20
        cap = int(math.ceil(1.12 * B / T))
        tgt = int(round(0.393 * cap))
        specs.append(dict(name=f"chain{c}", nx=side, ny=side, nz=side, S=S, T=T, cap_blocks=cap,
                          target_blocks=tgt, n_moves=n, shift_frac=0.5, seed=seed, mean=1.0,
                          cv=0.8, rng_a=5.0, nugget=0.1, sill=1.0))
    return specs


def chain_problem(spec: dict) -> Problem:
    """The Problem of one chain spec (see batched_chain_specs); spec keys may be
    overridden by the caller for smaller test cases."""
    kw = {k: spec[k] for k in ("name", "nx", "ny", "nz", "S", "T", "cap_blocks", "target_blocks", "n_moves",
                               "shift_frac", "seed", "mean", "cv", "rng_a", "nugget", "sill")}
    return make_problem(**kw)


def relaxed_x(B: int, T: int, seed: int) -> np.ndarray:
    """Fractional schedule x[b][t] in [0,1], rows drawn from Dirichlet(1) (float32)."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    x = rng.dirichlet(np.ones(T), size=B)
    return np.ascontiguousarray(x, dtype=np.float32)


def uncertainty_weights(T: int, S: int, seed: int = 4) -> np.ndarray:
    """Synthetic uncertainty weights sigma(s,t) of Eq. 12, float64 [T][S].

    Built as the product of Eq. 2: a spatial factor per scenario from Eq. 10,
    1 - I_s + sigma_local_s with Moran's I_s ~ U(0.2, 0.6) and local variance
    sigma_local_s ~ U(0.05, 0.3); a temporal confidence decay exp(-0.05 t);
    and a geological factor per (s, t) ~ U(0.9, 1.1) standing in for the
    feature-weighted term of Eq. 11 (so the weights are not a rank-one
    product).  Values lie in about [0.15, 1.2]."""
    rng = np.random.default_rng(np.random.SeedSequence(seed))
    moran = rng.uniform(0.2, 0.6, size=S)
    local = rng.uniform(0.05, 0.3, size=S)
    geo = rng.uniform(0.9, 1.1, size=(T, S))
    temporal = np.exp(-0.05 * np.arange(T, dtype=np.float64))
    return np.ascontiguousarray(temporal[:, None] * (1.0 - moran + local)[None, :] * geo, np.float64)
