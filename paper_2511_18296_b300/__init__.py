"""Python binding of the B300 move-evaluation engine (libmm.so, C ABI in mm.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  PyTorch supplies device memory and the stream.  If the library is
missing the import fails loudly; there is no CPU fallback.

Typical use::

    m = Model.from_problem(prob)          # grades, masses, economics -> device
    m.schedule_set(prob.x0)
    moves = torch.as_tensor(prob.moves, device="cuda")
    score, feas, mean = m.eval_moves(moves)
    idx, top, count = m.topk(score, feas, k=32)
    m.apply_move(tuple(prob.moves[int(idx[0])]))
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmm.so")

MM_OK = 0
STATUS = {0: "MM_OK", 1: "MM_ERR_INVALID_ARG", 2: "MM_ERR_CUDA", 3: "MM_ERR_OOM", 4: "MM_ERR_OVERFLOW",
          5: "MM_ERR_INFEASIBLE", 6: "MM_ERR_BAD_MOVE", 7: "MM_ERR_TIMEOUT", 8: "MM_ERR_STATE"}
MM_EVAL_PLAIN = 0
MM_EVAL_KAHAN = 1
MM_EVAL_GENERIC = 2
TOPK_MAX = 1024


class MMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MMModelDesc(C.Structure):
    _fields_ = [
        ("n_blocks", C.c_int32), ("n_scenarios", C.c_int32), ("n_periods", C.c_int32),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("pred_ptr", C.c_void_p), ("pred_idx", C.c_void_p),
        ("mass_t", C.c_void_p), ("grade", C.c_void_p),
        ("cap_t", C.c_void_p), ("mill_target_t", C.c_void_p),
        ("price", C.c_double), ("recovery", C.c_double),
        ("mining_cost", C.c_double), ("proc_cost", C.c_double),
        ("shortfall_pen", C.c_double), ("excess_pen", C.c_double),
        ("discount_rate", C.c_double), ("lam", C.c_double),
        ("sigma", C.c_void_p),
        ("cuda_stream", C.c_void_p),
    ]


class MMMove(C.Structure):
    _fields_ = [("b1", C.c_int32), ("arg", C.c_int32)]


class MMChain(C.Structure):
    _fields_ = [("model", C.c_void_p), ("moves_dev", C.c_void_p), ("n_moves", C.c_int64),
                ("score_dev", C.c_void_p), ("feasible_dev", C.c_void_p), ("idx_dev", C.c_void_p),
                ("topscore_dev", C.c_void_p), ("count_dev", C.c_void_p)]


_lib = None

# (name, restype, argtypes): every entry point declared in include/mm.h
P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
SIGNATURES = [
    ("mm_model_create", C.c_int, [P, P]),
    ("mm_model_destroy", None, [P]),
    ("mm_set_stream", C.c_int, [P, P]),
    ("mm_schedule_set", C.c_int, [P, P, P]),
    ("mm_schedule_get", C.c_int, [P, P]),
    ("mm_eval_moves", C.c_int, [P, P, I64, P, P, P]),
    ("mm_eval_moves_ex", C.c_int, [P, P, I64, P, P, P, P, I32]),
    ("mm_eval_violation", C.c_int, [P, P, I64, P, P]),
    ("mm_unpack_moves", C.c_int, [P, P, I64, P]),
    ("mm_relaxed_move_prior", C.c_int, [P, P, P, I64, P]),
    ("mm_set_tile", C.c_int, [P, I32, I32, I32, I32]),
    ("mm_topk", C.c_int, [P, P, P, I64, I32, P, P, P]),
    ("mm_topk_noalloc", C.c_int, [P, P, I64, I32, P, P, P, P]),
    ("mm_search_step", C.c_int, [P, P, I64, I32, I32, P, P, P, P, P]),
    ("mm_search_step_packed", C.c_int, [P, P, I64, I32, I32, P, P, P, P, P]),
    ("mm_set_step_event", C.c_int, [P, P]),
    ("mm_set_fp32_shadow", C.c_int, [P, I32]),
    ("mm_get_fp32_shadow_npv", C.c_int, [P, P]),
    ("mm_relaxed_forward", C.c_int, [P, P, P, D, D, P, P, P]),
    ("mm_relaxed_backward", C.c_int, [P, P, P, D, D, P, P, P, P, P]),
    ("mm_batch_create", C.c_int, [P, I32, I32, I32, P, P]),
    ("mm_batch_destroy", None, [P]),
    ("mm_batch_run", C.c_int, [P]),
    ("mm_batch_set_tile", C.c_int, [P, I32, I32]),
    ("mm_batch_get_tile", C.c_int, [P, P, P, P]),
    ("mm_batch_autotune", C.c_int, [P, I32, P, P, P]),
    ("mm_batch_set_chain", C.c_int, [P, I32, I32, I32]),
    ("mm_batch_get_chain", C.c_int, [P, I32, P, P]),
    ("mm_apply_move", C.c_int, [P, MMMove, P, P]),
    ("mm_apply_best", C.c_int, [P, P, I64, P, P]),
    ("mm_last_apply", C.c_int, [P, P, P, P]),
    ("mm_npv", C.c_int, [P, P, P, P]),
    ("mm_model_info", C.c_int, [P, P, P, P, P]),
    ("mm_get_ore", C.c_int, [P, P]),
    ("mm_get_values", C.c_int, [P, P]),
    ("mm_get_tonnage", C.c_int, [P, P, P]),
    ("mm_get_metal", C.c_int, [P, P]),
    ("mm_last_error", C.c_char_p, []),
]


def lib():
    """Load libmm.so (built by build.py); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run paper_2511_18296_b300/build.py)")
    l = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        f = getattr(l, name)
        f.restype = res
        f.argtypes = args
    _lib = l
    return l


def _check(st: int):
    if st != MM_OK:
        raise MMError(st, lib().mm_last_error().decode())


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def topk_noalloc(score, feas, k: int, idx, top, count, stream=None):
    """mm_topk_noalloc: top-k without any device allocation (caller passes
    every output buffer; the scratch is a fixed array inside the library).
    score float32 [n], feas uint8 [>= n], idx int32 [>= k], top float32
    [>= k], count int32 [>= 1]: contiguous CUDA tensors on one device
    (ValueError otherwise, before any device work)."""
    import torch
    n = int(score.shape[0])
    want = ((score, torch.float32, n, "score"), (feas, torch.uint8, n, "feas"), (idx, torch.int32, k, "idx"),
            (top, torch.float32, k, "top"), (count, torch.int32, 1, "count"))
    for t, dt, size, name in want:
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"topk_noalloc: {name} must be a contiguous CUDA tensor of {dt}")
        if t.numel() < size:
            raise ValueError(f"topk_noalloc: {name} holds {t.numel()} elements, needs {size}")
        if t.device != score.device:
            raise ValueError(f"topk_noalloc: {name} is on {t.device}, score on {score.device}")
    _check(lib().mm_topk_noalloc(_ptr(score), _ptr(feas), n, int(k), _ptr(idx), _ptr(top),
                                 _ptr(count), _stream_handle(stream)))
    return idx, top, count


def pack_moves(moves, B: int, T: int) -> np.ndarray:
    """Host-side compact form of a move batch for mm_unpack_moves: uint32
    (b1 << 16) | code, code = the swap partner, or 65535 - t for a shift to
    period t.  Needs B + T + 1 <= 65536 and valid moves (checked here)."""
    mv = np.asarray(moves, dtype=np.int64).reshape(-1, 2)
    if B + T + 1 > 65536:
        raise ValueError(f"packed moves need B + T + 1 <= 65536 (B = {B}, T = {T})")
    b1, arg = mv[:, 0], mv[:, 1]
    if ((b1 < 0) | (b1 >= B)).any() or ((arg >= B) | (arg < -(T + 1))).any():
        raise ValueError("a move is out of range for this model")
    code = np.where(arg >= 0, arg, 65535 - (-arg - 1))
    return np.ascontiguousarray(((b1 << 16) | code).astype(np.uint32))


class Model:
    """One block model on the device (owns an mm_model*)."""

    def __init__(self, B: int, S: int, T: int, mass, grade, cap, target, price: float, recovery: float,
                 mining_cost: float, proc_cost: float, shortfall_pen: float, excess_pen: float,
                 discount_rate: float, lam: float, grid: Optional[Tuple[int, int, int]] = None,
                 preds: Optional[Tuple[np.ndarray, np.ndarray]] = None, stream=None, sigma=None):
        """sigma: optional float64 [T][S] uncertainty weights sigma(s,t) of Eq. 12
        on the ore processing margin (see mm_model_desc.sigma)."""
        L = lib()
        self._keep = dict(mass=_np(mass, np.uint32), grade=_np(grade, np.float64).reshape(B, S),
                          cap=_np(cap, np.uint64), target=_np(target, np.uint64))
        if sigma is not None:
            self._keep["sigma"] = _np(sigma, np.float64).reshape(T, S)
        nx = ny = nz = 0
        pp = pi = None
        if grid is not None:
            nx, ny, nz = grid
        else:
            self._keep["pp"] = pp = _np(preds[0], np.int32)
            self._keep["pi"] = pi = _np(preds[1] if len(preds[1]) else np.zeros(1), np.int32)
        k = self._keep
        self.desc = MMModelDesc(B, S, T, nx, ny, nz,
                                pp.ctypes.data if pp is not None else None,
                                pi.ctypes.data if pi is not None else None,
                                k["mass"].ctypes.data, k["grade"].ctypes.data, k["cap"].ctypes.data,
                                k["target"].ctypes.data, price, recovery, mining_cost, proc_cost, shortfall_pen,
                                excess_pen, discount_rate, lam,
                                k["sigma"].ctypes.data if sigma is not None else None, _stream_handle(stream))
        h = C.c_void_p()
        _check(L.mm_model_create(C.byref(self.desc), C.byref(h)))
        self.h = h
        self.B, self.S, self.T = B, S, T
        self.weighted = sigma is not None
        self._keep = None  # the library copied everything it needs
        sp = C.c_int32()
        _check(L.mm_model_info(self.h, None, None, None, C.byref(sp)))
        self.S_pad = sp.value

    @classmethod
    def from_problem(cls, p, preds=None, stream=None, sigma=None) -> "Model":
        """From a workloads.Problem (1-5 grid unless a predecessor CSR is given)."""
        return cls(p.B, p.S, p.T, p.mass, p.grade, p.cap, p.target, p.price, p.recovery, p.mining_cost,
                   p.proc_cost, p.shortfall_pen, p.excess_pen, p.discount_rate, p.lam,
                   grid=None if preds is not None else (p.nx, p.ny, p.nz), preds=preds, stream=stream, sigma=sigma)

    def close(self):
        if getattr(self, "h", None):
            lib().mm_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile(self, team: int = 0, ctas_per_sm: int = 0, stages: int = -1, prefetch: int = -1):
        _check(lib().mm_set_tile(self.h, team, ctas_per_sm, stages, prefetch))

    def set_stream(self, stream=None):
        _check(lib().mm_set_stream(self.h, _stream_handle(stream)))

    # -- schedule -------------------------------------------------------
    def schedule_set(self, period) -> bool:
        x = _np(period, np.uint8)
        assert x.shape == (self.B,)
        feas = C.c_int()
        _check(lib().mm_schedule_set(self.h, x.ctypes.data, C.byref(feas)))
        return bool(feas.value)

    def schedule_get(self) -> np.ndarray:
        x = np.zeros(self.B, np.uint8)
        _check(lib().mm_schedule_get(self.h, x.ctypes.data))
        return x

    # -- evaluation -----------------------------------------------------
    def eval_moves(self, moves, score=None, feas=None, mean=None, want_mean=True, delta=None,
                   kahan: bool = False, generic: bool = False):
        """moves: int32 CUDA tensor [n, 2].  Returns (score f32, feasible u8, mean f32 or None)."""
        import torch
        assert moves.is_cuda and moves.dtype == torch.int32 and moves.is_contiguous()
        n = moves.shape[0]
        dev = moves.device
        if score is None:
            score = torch.empty(n, dtype=torch.float32, device=dev)
        if feas is None:
            feas = torch.empty(n, dtype=torch.uint8, device=dev)
        if mean is None and want_mean:
            mean = torch.empty(n, dtype=torch.float32, device=dev)
        L = lib()
        opts = (MM_EVAL_KAHAN if kahan else MM_EVAL_PLAIN) | (MM_EVAL_GENERIC if generic else 0)
        if delta is None and opts == 0:
            _check(L.mm_eval_moves(self.h, _ptr(moves), n, _ptr(score), _ptr(feas), _ptr(mean)))
        else:
            _check(L.mm_eval_moves_ex(self.h, _ptr(moves), n, _ptr(score), _ptr(feas), _ptr(mean), _ptr(delta),
                                      opts))
        return score, feas, mean

    def unpack_moves(self, packed, out=None):
        """mm_unpack_moves: uint32 packed moves (device) -> int32 [n, 2] moves (device)."""
        import torch
        assert packed.is_cuda and packed.dtype in (torch.int32, torch.uint32) and packed.is_contiguous()
        n = packed.shape[0]
        if out is None:
            out = torch.empty((n, 2), dtype=torch.int32, device=packed.device)
        _check(lib().mm_unpack_moves(self.h, _ptr(packed), n, _ptr(out)))
        return out

    def eval_violation(self, moves, cap_excess=None, prec_excess=None):
        """mm_eval_violation: (capacity excess int64 [n] in tonnes, precedence
        excess int32 [n] in periods) of each move; both 0 iff its flag is 1."""
        import torch
        assert moves.is_cuda and moves.dtype == torch.int32 and moves.is_contiguous()
        n = moves.shape[0]
        if cap_excess is None:
            cap_excess = torch.empty(n, dtype=torch.int64, device=moves.device)
        if prec_excess is None:
            prec_excess = torch.empty(n, dtype=torch.int32, device=moves.device)
        _check(lib().mm_eval_violation(self.h, _ptr(moves), n, _ptr(cap_excess), _ptr(prec_excess)))
        return cap_excess, prec_excess

    def eval_deltas(self, moves, kahan: bool = False, generic: bool = False):
        """Per-scenario deltas [n, S] as well (parity/debug path)."""
        import torch
        delta = torch.empty((moves.shape[0], self.S), dtype=torch.float32, device=moves.device)
        score, feas, mean = self.eval_moves(moves, delta=delta, kahan=kahan, generic=generic)
        return score, feas, mean, delta

    def topk(self, score, feas, k: int, idx=None, top=None, count=None):
        import torch
        n = score.shape[0]
        dev = score.device
        if idx is None:
            idx = torch.empty(k, dtype=torch.int32, device=dev)
        if top is None:
            top = torch.empty(k, dtype=torch.float32, device=dev)
        if count is None:
            count = torch.empty(1, dtype=torch.int32, device=dev)
        _check(lib().mm_topk(self.h, _ptr(score), _ptr(feas), n, k, _ptr(idx), _ptr(top), _ptr(count)))
        return idx, top, count

    def search_step(self, moves, k: int = 32, apply: bool = True, score=None, feas=None, idx=None, top=None,
                    count=None):
        """Evaluate + top-k (k <= 32) + optional device apply of the best move, one launch."""
        import torch
        n = moves.shape[0]
        dev = moves.device
        if score is None:
            score = torch.empty(n, dtype=torch.float32, device=dev)
        if feas is None:
            feas = torch.empty(n, dtype=torch.uint8, device=dev)
        if idx is None:
            idx = torch.empty(k, dtype=torch.int32, device=dev)
        if top is None:
            top = torch.empty(k, dtype=torch.float32, device=dev)
        if count is None:
            count = torch.empty(1, dtype=torch.int32, device=dev)
        _check(lib().mm_search_step(self.h, _ptr(moves), n, k, 1 if apply else 0, _ptr(score), _ptr(feas), _ptr(idx),
                                    _ptr(top), _ptr(count)))
        return score, feas, idx, top, count

    def search_step_packed(self, packed, k: int = 32, apply: bool = True, score=None, feas=None, idx=None, top=None,
                           count=None):
        """mm_search_step_packed: search_step on a batch in the compact 4-byte
        form (pack_moves), decoded inside the evaluation launch."""
        import torch
        assert packed.is_cuda and packed.dtype in (torch.int32, torch.uint32) and packed.is_contiguous()
        n = packed.shape[0]
        dev = packed.device
        if score is None:
            score = torch.empty(n, dtype=torch.float32, device=dev)
        if feas is None:
            feas = torch.empty(n, dtype=torch.uint8, device=dev)
        if idx is None:
            idx = torch.empty(k, dtype=torch.int32, device=dev)
        if top is None:
            top = torch.empty(k, dtype=torch.float32, device=dev)
        if count is None:
            count = torch.empty(1, dtype=torch.int32, device=dev)
        _check(lib().mm_search_step_packed(self.h, _ptr(packed), n, k, 1 if apply else 0, _ptr(score), _ptr(feas),
                                           _ptr(idx), _ptr(top), _ptr(count)))
        return score, feas, idx, top, count

    def set_step_event(self, event=None):
        """Timing hook: record `event` (a timing-enabled torch.cuda.Event that
        has been recorded once, or a raw cudaEvent_t) between the two launches
        of every later search_step; None turns it off."""
        h = None
        if event is not None:
            h = event.cuda_event if hasattr(event, "cuda_event") else int(event)
            if not h:
                raise ValueError("the event has no CUDA handle yet (record it once first)")
        self._step_event = event  # keep the caller's event alive while it is in use
        _check(lib().mm_set_step_event(self.h, h))

    # -- precision study -------------------------------------------------
    def set_fp32_shadow(self, enable: bool = True):
        _check(lib().mm_set_fp32_shadow(self.h, 1 if enable else 0))

    def fp32_shadow_npv(self) -> np.ndarray:
        v = np.zeros(self.S, np.float64)
        _check(lib().mm_get_fp32_shadow_npv(self.h, v.ctypes.data))
        return v

    # -- relaxed objective ------------------------------------------------
    def relaxed_move_prior(self, gx, moves, prior=None):
        """mm_relaxed_move_prior: first-order change of the relaxed J for each
        move at the current schedule, from gx = dJ/dx [B, T] (device)."""
        import torch
        n = moves.shape[0]
        if prior is None:
            prior = torch.empty(n, dtype=torch.float32, device=moves.device)
        _check(lib().mm_relaxed_move_prior(self.h, _ptr(gx), _ptr(moves), n, _ptr(prior)))
        return prior

    def relaxed_forward(self, x, g=None, beta: float = 10.0, m_ref: float = 10_000.0):
        """J (float64 [1]), NPV_s (float64 [S]) and the checkpoint O[t][s]
        (float64 [T][S]) of the relaxed objective for x float32 [B][T] (CUDA);
        g float32 [B][S] (CUDA) or None for the model's own grades."""
        import torch
        dev = x.device
        J = torch.empty(1, dtype=torch.float64, device=dev)
        npv = torch.empty(self.S, dtype=torch.float64, device=dev)
        ot = torch.empty((self.T, self.S), dtype=torch.float64, device=dev)
        _check(lib().mm_relaxed_forward(self.h, _ptr(x), _ptr(g), beta, m_ref, _ptr(J), _ptr(npv), _ptr(ot)))
        return J, npv, ot

    def relaxed_backward(self, x, g, npv, ot, gJ, beta: float = 10.0, m_ref: float = 10_000.0, want_g: bool = True):
        """dJ/dx float32 [B][T] and dJ/dg float32 [B][S] (None unless want_g)."""
        import torch
        gx = torch.empty_like(x)
        gg = torch.empty((self.B, self.S), dtype=torch.float32, device=x.device) if want_g else None
        _check(lib().mm_relaxed_backward(self.h, _ptr(x), _ptr(g), beta, m_ref, _ptr(npv), _ptr(ot), _ptr(gJ),
                                         _ptr(gx), _ptr(gg)))
        return gx, gg

    # -- apply ----------------------------------------------------------
    def apply_move(self, move) -> Tuple[float, float]:
        """Apply (b1, arg); returns the NPV (mean, std).  Raises MMError with
        MM_ERR_INFEASIBLE / MM_ERR_BAD_MOVE (nothing changed)."""
        mean, sd = C.c_double(), C.c_double()
        _check(lib().mm_apply_move(self.h, MMMove(int(move[0]), int(move[1])), C.byref(mean), C.byref(sd)))
        return mean.value, sd.value

    def apply_best(self, moves, idx, count):
        _check(lib().mm_apply_best(self.h, _ptr(moves), int(moves.shape[0]), _ptr(idx), _ptr(count)))

    def last_apply(self):
        a, mean, sd = C.c_int32(), C.c_double(), C.c_double()
        _check(lib().mm_last_apply(self.h, C.byref(a), C.byref(mean), C.byref(sd)))
        return a.value, mean.value, sd.value

    # -- inspection -----------------------------------------------------
    def npv(self):
        v = np.zeros(self.S, np.float64)
        mean, sd = C.c_double(), C.c_double()
        _check(lib().mm_npv(self.h, v.ctypes.data, C.byref(mean), C.byref(sd)))
        return v, mean.value, sd.value

    def ore_bits(self) -> np.ndarray:
        """uint8 [B][S] ore flags unpacked from the device bitmask."""
        W = (self.S + 31) // 32
        w = np.zeros((self.B, W), np.uint32)
        _check(lib().mm_get_ore(self.h, w.ctypes.data))
        bits = np.unpackbits(w.view(np.uint8).reshape(self.B, W * 4), axis=1, bitorder="little")
        return bits[:, :self.S]

    def values(self) -> np.ndarray:
        v = np.zeros((self.B, self.S), np.float32)
        _check(lib().mm_get_values(self.h, v.ctypes.data))
        return v

    def tonnage(self):
        mined = np.zeros(self.T, np.int64)
        oreT = np.zeros((self.T, self.S), np.int64)
        _check(lib().mm_get_tonnage(self.h, mined.ctypes.data, oreT.ctypes.data))
        return mined, oreT

    def metal(self) -> np.ndarray:
        m = np.zeros((self.T, self.S), np.float64)
        _check(lib().mm_get_metal(self.h, m.ctypes.data))
        return m


class Batch:
    """Many chains evaluated in one persistent launch (mm_batch_*).

    chains: list of (model, moves) with moves an int32 [n, 2] CUDA tensor; the
    batch allocates each chain's outputs (score, feas, idx, top, count) and
    keeps references to every buffer it was given."""

    def __init__(self, chains, k: int = 32, apply: bool = False, stream=None):
        import torch
        self.k = k
        self.models = [m for m, _ in chains]
        self.moves = [mv for _, mv in chains]
        self.out = []
        arr = (MMChain * len(chains))()
        for i, (m, mv) in enumerate(chains):
            n = int(mv.shape[0])
            dev = mv.device
            o = dict(score=torch.empty(n, dtype=torch.float32, device=dev),
                     feas=torch.empty(n, dtype=torch.uint8, device=dev),
                     idx=torch.empty(k, dtype=torch.int32, device=dev),
                     top=torch.empty(k, dtype=torch.float32, device=dev),
                     count=torch.empty(1, dtype=torch.int32, device=dev))
            self.out.append(o)
            mh = m.h.value if isinstance(m.h, C.c_void_p) else m.h
            arr[i] = MMChain(mh, _ptr(mv), n, _ptr(o["score"]), _ptr(o["feas"]), _ptr(o["idx"]), _ptr(o["top"]),
                             _ptr(o["count"]))
        self.stream = stream
        h = C.c_void_p()
        _check(lib().mm_batch_create(arr, len(chains), k, 1 if apply else 0, _stream_handle(stream), C.byref(h)))
        self.h = h

    def run(self):
        _check(lib().mm_batch_run(self.h))

    def set_tile(self, moves_per_item: int, ctas_per_sm: int = 0):
        _check(lib().mm_batch_set_tile(self.h, moves_per_item, ctas_per_sm))

    def tile(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().mm_batch_get_tile(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def set_chain(self, chain: int, team: int = 0, prefetch: int = -1):
        _check(lib().mm_batch_set_chain(self.h, chain, team, prefetch))

    def chain_shape(self, chain: int):
        a, b = C.c_int32(), C.c_int32()
        _check(lib().mm_batch_get_chain(self.h, chain, C.byref(a), C.byref(b)))
        return a.value, b.value

    def chain_key(self, chain: int) -> str:
        """The key a chain's tuned shape is stored under: its scenario count,
        block count and move count."""
        m = self.models[chain]
        return f"S{m.S}_B{m.B}_n{int(self.moves[chain].shape[0])}"

    def autotune(self, reps: int = 3, cache: Optional[str] = None):
        """mm_batch_autotune: tile shape, then team width per scenario count,
        then prefetch distance per scenario count.  Returns (moves per item,
        CTAs per SM, best ms).

        cache: a JSON file of earlier choices (default: $MM_BATCH_TUNE_CACHE,
        none when unset).  Each chain's team width and prefetch distance are
        stored under its (S, B, n) key and the tile under the sorted list of
        the batch's chain keys; when every key of this batch is present the
        stored choices are installed without timing anything (the returned
        time is the stored one)."""
        import hashlib
        import json
        path = cache if cache is not None else os.environ.get("MM_BATCH_TUNE_CACHE")
        keys = [self.chain_key(i) for i in range(len(self.models))]
        tile_key = "tile_" + hashlib.sha1(",".join(sorted(keys)).encode()).hexdigest()[:16]
        data = {"chains": {}, "tiles": {}}
        if path and os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
            chains, tiles = data.get("chains", {}), data.get("tiles", {})
            if tile_key in tiles and all(k in chains for k in keys):
                t = tiles[tile_key]
                self.set_tile(t["moves_per_item"], t["ctas_per_sm"])
                for i, k in enumerate(keys):
                    self.set_chain(i, chains[k]["team"], chains[k]["prefetch"])
                return t["moves_per_item"], self.tile()[1], t["ms"]
        a, b, ms = C.c_int32(), C.c_int32(), C.c_float()
        _check(lib().mm_batch_autotune(self.h, reps, C.byref(a), C.byref(b), C.byref(ms)))
        if path:
            data.setdefault("chains", {})
            data.setdefault("tiles", {})
            for i, k in enumerate(keys):
                team, pf = self.chain_shape(i)
                data["chains"][k] = {"team": team, "prefetch": pf}
            data["tiles"][tile_key] = {"moves_per_item": a.value, "ctas_per_sm": b.value, "ms": ms.value}
            tmp = path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        return a.value, b.value, ms.value

    def close(self):
        if getattr(self, "h", None):
            lib().mm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _relaxed_function():
    import torch

    class RelaxedObjective(torch.autograd.Function):
        """J = mean_s NPV_s - lambda std_s NPV_s of the relaxed schedule x
        (float32 [B][T]) and grades g (float32 [B][S]) on a model; backward runs
        the library's adjoint kernels (dJ/dx, dJ/dg).  The forward keeps the
        per-period checkpoint O[t][s] for the backward."""

        @staticmethod
        def forward(ctx, x, g, model, beta, m_ref):
            x = x.contiguous()
            g = g.contiguous()
            J, npv, ot = model.relaxed_forward(x, g, beta, m_ref)
            ctx.save_for_backward(x, g, npv, ot)
            ctx.model, ctx.beta, ctx.m_ref = model, beta, m_ref
            return J[0]

        @staticmethod
        def backward(ctx, gJ):
            x, g, npv, ot = ctx.saved_tensors
            gJ = gJ.reshape(1).to(torch.float64).contiguous()
            gx, gg = ctx.model.relaxed_backward(x, g, npv, ot, gJ, ctx.beta, ctx.m_ref, want_g=ctx.needs_input_grad[1])
            return gx, gg, None, None, None

    return RelaxedObjective


_RELAXED = None


def relaxed_objective(model, x, g, beta: float = 10.0, m_ref: float = 10_000.0):
    """Differentiable J(x, g) through torch.autograd (float64 scalar tensor)."""
    global _RELAXED
    if _RELAXED is None:
        _RELAXED = _relaxed_function()
    return _RELAXED.apply(x, g, model, beta, m_ref)
