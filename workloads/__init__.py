"""Seeded synthetic inputs for the move-evaluation engine and for the oracle.

This package builds inputs only: block grids, lognormal grade scenarios from a
Gaussian random field, an initial schedule and random candidate moves.  It holds
none of the evaluation arithmetic (no ore/waste rule, no values, no discounting,
no penalties, no feasibility test), so the CUDA path and the oracle can both
consume its output without sharing any of the method's code.

The stand-in for the paper's deposits: the paper's block models and its
VAE-generated scenarios (Section 5.3) are not public, so grades come from a
Gaussian random field with an exponential variogram, exponentiated to a
lognormal, which is the shock model the paper names for its own Monte Carlo
study (Section 7.1.3).
"""

from .grf import lognormal_grades, gaussian_field
from .configs import (
    Problem,
    make_problem,
    chain_problem,
    greedy_schedule,
    random_moves,
    CONFIGS,
    config,
    batched_chain_specs,
    relaxed_x,
    uncertainty_weights,
)

__all__ = [
    "lognormal_grades",
    "gaussian_field",
    "Problem",
    "make_problem",
    "greedy_schedule",
    "random_moves",
    "CONFIGS",
    "config",
    "batched_chain_specs",
    "relaxed_x",
    "uncertainty_weights",
]
