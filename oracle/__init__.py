"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, FP64,
OpenMP over moves) with ctypes and shares no code with the CUDA library.

Functions follow the problem statement of the paper: Eq. 14 (objective),
Eq. 15 (precedence), Eq. 16 (capacity), the ore/waste reading of Eq. 18, and the
candidate moves of Algorithms 4-5.  The relaxed (fractional) objective lives in
``oracle.relaxed`` as float64 PyTorch CPU code.

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, hand-computed fixtures in ``tests/golden/``, a library
transitive closure (networkx), brute-force enumeration and invariants.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "liboracle.so")
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        from .build import build
        build()
    lib = C.CDLL(_LIB_PATH)
    P = C.c_void_p
    lib.or_num_threads.restype = C.c_int
    lib.or_stencil_preds.restype = C.c_int64
    lib.or_stencil_preds.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, P]
    lib.or_classify.argtypes = [P, P, P]
    lib.or_tonnage.argtypes = [P, P, P, P, P]
    lib.or_npv.argtypes = [P, P, P, P, P]
    lib.or_feasible.restype = C.c_int
    lib.or_feasible.argtypes = [P, P]
    lib.or_eval_bruteforce.argtypes = [P, P, P, P, P, C.c_int64, P, P, P, P, P]
    lib.or_eval_incremental.argtypes = [P, P, P, P, P, C.c_int64, P, P, P, P, P, P, P]
    lib.or_topk.restype = C.c_int32
    lib.or_topk.argtypes = [P, P, C.c_int64, C.c_int32, P, P]
    lib.or_apply.restype = C.c_int
    lib.or_apply.argtypes = [P, P, C.c_int32, C.c_int32]
    lib.or_violation.argtypes = [P, P, P, C.c_int64, P, P]
    _lib = lib
    return lib


class _OrModel(C.Structure):
    _fields_ = [
        ("B", C.c_int32), ("S", C.c_int32), ("T", C.c_int32),
        ("pred_ptr", C.c_void_p), ("pred_idx", C.c_void_p),
        ("mass", C.c_void_p), ("grade", C.c_void_p),
        ("cap", C.c_void_p), ("target", C.c_void_p),
        ("price", C.c_double), ("recovery", C.c_double),
        ("mining_cost", C.c_double), ("proc_cost", C.c_double),
        ("shortfall_pen", C.c_double), ("excess_pen", C.c_double),
        ("discount_rate", C.c_double), ("lam", C.c_double),
        ("sigma", C.c_void_p),
    ]


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    return int(_load().or_num_threads())


def stencil_preds(nx: int, ny: int, nz: int):
    """CSR (ptr[B+1], idx[E]) of the 1-5 predecessor pattern."""
    lib = _load()
    B = nx * ny * nz
    E = lib.or_stencil_preds(nx, ny, nz, None, None)
    ptr = np.zeros(B + 1, np.int32)
    idx = np.zeros(max(E, 1), np.int32)
    lib.or_stencil_preds(nx, ny, nz, _p(ptr), _p(idx))
    return ptr, idx[:E]


class OracleModel:
    """FP64 oracle over one problem instance (a ``workloads.Problem`` or any
    object with the same attributes).  ``preds`` overrides the 1-5 stencil with
    an explicit CSR (ptr, idx) of direct predecessors.  ``sigma`` (float64
    [T][S], optional) holds the uncertainty weights sigma(s,t) of Eq. 12, which
    scale the processing margin of ore blocks."""

    def __init__(self, prob, preds=None, sigma=None):
        self.lib = _load()
        self.B, self.S, self.T = prob.B, prob.S, prob.T
        if preds is None:
            preds = stencil_preds(prob.nx, prob.ny, prob.nz)
        self.pred_ptr = np.ascontiguousarray(preds[0], np.int32)
        self.pred_idx = np.ascontiguousarray(preds[1] if len(preds[1]) else np.zeros(1, np.int32), np.int32)
        self.mass = np.ascontiguousarray(prob.mass, np.uint32)
        self.grade = np.ascontiguousarray(prob.grade, np.float64).reshape(self.B, self.S)
        self.cap = np.ascontiguousarray(prob.cap, np.uint64)
        self.target = np.ascontiguousarray(prob.target, np.uint64)
        self.m = _OrModel(self.B, self.S, self.T, _p(self.pred_ptr), _p(self.pred_idx), _p(self.mass),
                          _p(self.grade), _p(self.cap), _p(self.target), prob.price, prob.recovery,
                          prob.mining_cost, prob.proc_cost, prob.shortfall_pen, prob.excess_pen,
                          prob.discount_rate, prob.lam, None)
        self.sigma = None
        if sigma is not None:
            self.sigma = np.ascontiguousarray(sigma, np.float64).reshape(self.T, self.S)
            self.m.sigma = _p(self.sigma)
        self.ore, self.value = self.classify()

    @property
    def _mp(self):
        return C.byref(self.m)

    def classify(self):
        ore = np.zeros((self.B, self.S), np.uint8)
        val = np.zeros((self.B, self.S), np.float64)
        self.lib.or_classify(self._mp, _p(ore), _p(val))
        return ore, val

    def tonnage(self, x):
        x = np.ascontiguousarray(x, np.uint8)
        mined = np.zeros(self.T, np.int64)
        oreT = np.zeros((self.T, self.S), np.int64)
        self.lib.or_tonnage(self._mp, _p(self.ore), _p(x), _p(mined), _p(oreT))
        return mined, oreT

    def npv(self, x):
        x = np.ascontiguousarray(x, np.uint8)
        out = np.zeros(self.S, np.float64)
        self.lib.or_npv(self._mp, _p(self.ore), _p(self.value), _p(x), _p(out))
        return out

    def feasible(self, x) -> bool:
        x = np.ascontiguousarray(x, np.uint8)
        return bool(self.lib.or_feasible(self._mp, _p(x)))

    def _outs(self, n, want_delta):
        return dict(
            delta=np.zeros((n, self.S), np.float64) if want_delta else None,
            mean=np.zeros(n, np.float64), std=np.zeros(n, np.float64),
            score=np.zeros(n, np.float64), flag=np.zeros(n, np.uint8))

    def eval_bruteforce(self, x, moves, want_delta=True):
        """Delta_s = NPV_s(x') - NPV_s(x) recomputed in full for every move."""
        x = np.ascontiguousarray(x, np.uint8)
        mv = np.ascontiguousarray(moves, np.int32).reshape(-1, 2)
        n = mv.shape[0]
        o = self._outs(n, want_delta)
        d = o["delta"]
        self.lib.or_eval_bruteforce(self._mp, _p(self.ore), _p(self.value), _p(x), _p(mv), n,
                                    _p(d) if d is not None else None, _p(o["mean"]), _p(o["std"]),
                                    _p(o["score"]), _p(o["flag"]))
        return o

    def eval_incremental(self, x, moves, want_delta=False, want_floor_s=False):
        """O(S)-per-move FP64 evaluator; also returns the per-move error-scale
        floor F (mean over scenarios of the magnitudes of the delta's terms)."""
        x = np.ascontiguousarray(x, np.uint8)
        mv = np.ascontiguousarray(moves, np.int32).reshape(-1, 2)
        n = mv.shape[0]
        o = self._outs(n, want_delta)
        o["floor"] = np.zeros(n, np.float64)
        o["floor_s"] = np.zeros((n, self.S), np.float64) if want_floor_s else None
        d, fs = o["delta"], o["floor_s"]
        self.lib.or_eval_incremental(self._mp, _p(self.ore), _p(self.value), _p(x), _p(mv), n,
                                     _p(d) if d is not None else None, _p(o["mean"]), _p(o["std"]),
                                     _p(o["score"]), _p(o["flag"]), _p(o["floor"]),
                                     _p(fs) if fs is not None else None)
        return o

    def violation(self, x, moves):
        """(capacity excess int64 [n] tonnes, precedence excess int32 [n]
        periods) of each move by brute force; -1 for bad moves."""
        xx = np.ascontiguousarray(x, np.uint8)
        mv = np.ascontiguousarray(moves, np.int32).reshape(-1, 2)
        n = mv.shape[0]
        ce = np.zeros(max(n, 1), np.int64)
        pe = np.zeros(max(n, 1), np.int32)
        self.lib.or_violation(self._mp, _p(xx), _p(mv), n, _p(ce), _p(pe))
        return ce[:n], pe[:n]

    def apply(self, x, move) -> int:
        """Apply (b1, arg) to x in place: 0 applied, 1 infeasible, 2 bad move."""
        assert x.dtype == np.uint8 and x.flags.c_contiguous
        return int(self.lib.or_apply(self._mp, _p(x), int(move[0]), int(move[1])))


def topk(score, flag, k: int):
    """(idx, score) of the k feasible moves with the largest score, ties to the
    lower index."""
    lib = _load()
    s = np.ascontiguousarray(score, np.float64)
    f = np.ascontiguousarray(flag, np.uint8)
    n = s.shape[0]
    idx = np.zeros(max(k, 1), np.int32)
    top = np.zeros(max(k, 1), np.float64)
    c = lib.or_topk(_p(s), _p(f), n, k, _p(idx), _p(top))
    return idx[:c], top[:c]


def risk_score(delta: np.ndarray, lam: float):
    """mean_s - lam * std_s (population std), row-wise, FP64."""
    mu = delta.mean(axis=1)
    sd = np.sqrt(((delta - mu[:, None]) ** 2).mean(axis=1))
    return mu - lam * sd
