"""Benchmark: move-scenario evaluations per second on the 50k-block workload.

One step = one pass of the whole hot path over one batch of moves resident in
HBM: mm_eval_moves (decode, exact feasibility, per-scenario NPV delta,
mean - lambda*std) -> mm_topk -> mm_apply_best (the best feasible move applied
on the device, FP64 accumulators updated).  Workload: 50x50x20 = 50,000 blocks,
S = 100 lognormal grade scenarios, T = 20 periods, 262,144 moves (half shifts,
half swaps), synthetic and seeded.  The value rows (21 MB) fit in L2, so L2 is
flushed (a 256 MB write, outside the per-step events) before every timed step.

Prints one JSON line (rank 0).  Arms:
  default           the CUDA path (value: device-timed; e2e: host buffers through
                    the C ABI, copies inside the timed region);
  --impl reference  the FP64 CPU oracle on the host cores (the only reference
                    arm available: the paper publishes no code).
Multi-GPU (torchrun): every rank evaluates its own independent batch on its own
GPU (no data-path collective); value = all ranks' evaluations / max rank time.
"""

from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "plain_50k"
METRIC = "move-scenario evals/sec at 50k blocks, S=100; % of HBM roofline vs plain form"
UNIT = "move-scenario evals/s"
TOPK = 32
HBM_NOMINAL_GBS = 7700.0  # B300 HBM3e nominal bandwidth, for context beside the measured copy peak
FLUSH_BYTES = 256 << 20
K_FORM = 50  # timed steps of every secondary form (median and best of 50)
EVAL_KERNEL = "k_eval_tiled"  # the move evaluator (mm_eval_moves launches it alone)
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_eval_tiled_plain_50k.md")
EVAL_SOURCES = ["paper_2511_18296_b300/csrc/mm_eval.cu", "paper_2511_18296_b300/csrc/mm_eval_tiled.cuh",
                "paper_2511_18296_b300/csrc/mm_eval_fast_plain.cu", "paper_2511_18296_b300/csrc/mm_apply.cuh",
                "paper_2511_18296_b300/csrc/mm_move.cuh", "paper_2511_18296_b300/csrc/mm_internal.cuh",
                "paper_2511_18296_b300/csrc/mm_sort.cuh"]


def algorithmic_bytes(moves: np.ndarray, S: int) -> float:
    """Bytes a move batch must touch at minimum: 8 (move) + 5 (score + flag) +
    per moved block (11 + 4S + S/8): its period byte and ten neighbour period
    bytes, an FP32 value row and an ore bit row."""
    n_swap = int((moves[:, 1] >= 0).sum())
    n_shift = moves.shape[0] - n_swap
    per_block = 11 + 4 * S + S / 8
    return n_shift * (13 + per_block) + n_swap * (13 + 2 * per_block)


def source_sha() -> str:
    h = hashlib.sha256()
    for f in EVAL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the evaluator from the committed ncu summary,
    or None when absent or taken on another version of the kernel source."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256_16") != source_sha():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def mark(self):
        return time.time()

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self, t0: float, t1: float):
        rows = []
        for r in csv.reader(io.StringIO(self.out)):
            if len(r) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(r[0].strip().split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + r[0].strip().split(".")[1]) if "." in r[0] else 0.0
            except Exception:
                continue
            rows.append((ts, [x.strip() for x in r]))
        inside = [r for ts, r in rows if t0 - 0.05 <= ts <= t1 + 0.05] or [r for _, r in rows]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in inside if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside),
                "power_w_max": max((float(r[4]) for r in inside if r[4].replace(".", "").isdigit()), default=None)}


class StepTimer:
    """Device time of single steps, each bracketed by two CUDA events recorded
    inside a CUDA graph (external event nodes), an L2 flush before every step
    outside the events.  A graph holds up to R steps; it is replayed until K
    steps are timed, reading its events after each replay (a replay re-records
    them).  The host enqueues nothing between the events, so host overhead never
    shows up inside a step."""

    def __init__(self, stream, flush, R: int = 50):
        self.stream, self.flush, self.R = stream, flush, R

    def graph(self, fns, R=None):
        import torch
        R = R or self.R
        evs = [(torch.cuda.Event(enable_timing=True, external=True),
                torch.cuda.Event(enable_timing=True, external=True)) for _ in range(R)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            for e0, e1 in evs:
                self.flush.zero_()
                e0.record(self.stream)
                for fn in fns:
                    fn()
                e1.record(self.stream)
        return g, evs

    def run(self, ge, K: int, between=None):
        """Per-step device times (ms) of K steps; between() (untimed) runs
        after every replay that another replay follows."""
        g, evs = ge
        out = []
        while len(out) < K:
            g.replay()
            evs[-1][1].synchronize()
            out.extend(e0.elapsed_time(e1) for e0, e1 in evs)
            if between is not None and len(out) < K:
                between()
        return out[:K]

    def warm(self, ge, seconds: float = 0.0, reps: int = 3):
        """Untimed replays: at least reps, and for at least `seconds` (brings the
        clocks up under load before a timed region)."""
        g, evs = ge
        t0 = time.perf_counter()
        r = 0
        while r < reps or time.perf_counter() - t0 < seconds:
            g.replay()
            r += 1
        evs[-1][1].synchronize()


def stats(ts):
    """Median, best, interquartile range and mean of per-step times (ms)."""
    a = np.asarray(ts, float)
    return {"n": int(a.size), "median_ms": float(np.median(a)), "min_ms": float(a.min()),
            "p25_ms": float(np.percentile(a, 25)), "p75_ms": float(np.percentile(a, 75)),
            "mean_ms": float(a.mean())}


# ----------------------------------------------------------------- CPU oracle


def cpu_baseline(p, budget_s: float = 12.0):
    """The FP64 oracle as it stands, on the host cores: the incremental
    evaluator over whole batches and the brute-force definition on a sample."""
    import oracle as O
    om = O.OracleModel(p)
    cores = O.num_threads()
    n = p.moves.shape[0]
    om.eval_incremental(p.x0, p.moves[:1024])
    t0 = time.perf_counter()
    reps = 0
    while True:
        om.eval_incremental(p.x0, p.moves)
        reps += 1
        if time.perf_counter() - t0 > budget_s * 0.6:
            break
    inc_rate = reps * n * p.S / (time.perf_counter() - t0)
    nb = 8
    t0 = time.perf_counter()
    done = 0
    while time.perf_counter() - t0 < budget_s * 0.4:
        om.eval_bruteforce(p.x0, p.moves[done % n:done % n + nb], want_delta=False)
        done += nb
    bf_rate = done * p.S / (time.perf_counter() - t0)
    return {"value": inc_rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"incremental FP64 evaluator: {reps} full batches of {n} moves x {p.S} scenarios; "
                      f"brute force (full NPV recompute per move): {done} moves",
            "bruteforce_value": bf_rate}


def accuracy_report(p, sel, gpu, k: int = 32):
    """Error of the GPU scores against the FP64 oracle's on a sample of the
    batch: the largest |gpu - ref| / max(|ref|, F) (F = the oracle's scale of
    the summed terms), whether the flags agree bit for bit, and whether the
    sample's top-k indices agree (ties within the bound allowed to swap)."""
    import oracle as O
    import workloads as W
    out = {"sample": f"{len(sel)} moves of the batch (seed 5) at the initial schedule", "bound": 1e-5}
    for form, sig in (("plain", None), ("compensated", None), ("weighted", W.uncertainty_weights(p.T, p.S))):
        om = O.OracleModel(p, sigma=sig)
        ref = om.eval_incremental(p.x0, p.moves[sel])
        score, flag = gpu[form]
        r, f = ref["score"], ref["floor"]
        ok = np.isfinite(r)
        err = np.abs(score[ok].astype(np.float64) - r[ok]) / np.maximum(np.abs(r[ok]), np.maximum(f[ok], 1e-300))
        gi, _ = O.topk(score.astype(np.float64), flag, k)
        ri, rtop = O.topk(r, ref["flag"], k)
        same = np.array_equal(gi, ri)
        if not same and len(gi) == len(ri):
            # a swap is allowed only inside a certified near-tie of the oracle's scores
            same = bool(np.all(np.abs(r[gi] - r[ri]) <= 1e-5 * np.maximum(np.abs(r[ri]), f[ri])))
        out[form] = {"max_rel_err": float(err.max()) if err.size else 0.0,
                     "flags_equal": bool(np.array_equal(flag, ref["flag"])), "topk_agrees": bool(same)}
    return out


def full_batch_accuracy(p, score, flag):
    """The plain form's scores of the whole batch at the initial schedule
    against the FP64 oracle's: largest relative error (to max(|ref|, F)),
    flags bit for bit, and for the top 32 and top 256 the number of index
    positions that differ from the oracle's selection, each of which must be a
    certified near-tie (the oracle's two scores within 1e-5 of each other)."""
    import oracle as O
    ref = O.OracleModel(p).eval_incremental(p.x0, p.moves)
    r, f = ref["score"], ref["floor"]
    ok = np.isfinite(r)
    err = np.abs(score[ok].astype(np.float64) - r[ok]) / np.maximum(np.abs(r[ok]), np.maximum(f[ok], 1e-300))
    out = {"moves": int(score.shape[0]), "max_rel_err": float(err.max()) if err.size else 0.0,
           "flags_equal": bool(np.array_equal(flag, ref["flag"])), "bound": 1e-5}
    for k in (32, 256):
        gi, _ = O.topk(score.astype(np.float64), flag, k)
        ri, _ = O.topk(r, ref["flag"], k)
        diff = np.nonzero(gi != ri)[0] if gi.size == ri.size else np.arange(max(gi.size, ri.size))
        certified = gi.size == ri.size and all(
            abs(r[gi[j]] - r[ri[j]]) <= 1e-5 * max(abs(r[gi[j]]), abs(r[ri[j]]), f[gi[j]], f[ri[j]]) for j in diff)
        out[f"top{k}"] = {"swaps": int(diff.size), "all_certified_near_ties": bool(certified)}
    return out


def drift_report(p, x_final, npv64, npv32, n_apply: int,
                 workload: str = "the bench batch, search steps with apply from the initial schedule"):
    """NPV_s of the device's running FP64 totals and of their FP32 shadow after
    n_apply applies, against the oracle's full FP64 recomputation of the same
    schedule: the largest relative difference over scenarios."""
    import oracle as O
    ref = O.OracleModel(p).npv(x_final)
    scale = np.maximum(np.abs(ref), 1.0)
    return {"applies": n_apply, "workload": workload,
            "fp64_running_max_rel": float(np.max(np.abs(npv64 - ref) / scale)),
            "fp32_shadow_max_rel": float(np.max(np.abs(npv32 - ref) / scale))}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    import workloads as W
    p = W.config(WORKLOAD)
    om = O.OracleModel(p)
    cores = O.num_threads()
    n_all = p.moves.shape[0]
    # size each step so that warm-up + timed steps take about a minute
    t0 = time.perf_counter()
    om.eval_incremental(p.x0, p.moves[:16384])
    per_move = (time.perf_counter() - t0) / 16384
    n = int(min(n_all, max(1024, 60.0 / max(args.steps + args.warmup, 1) / max(per_move, 1e-9))))
    x = p.x0.copy()

    def step(j):
        lo = (j * n) % n_all
        mv = p.moves[lo:lo + n] if lo + n <= n_all else np.concatenate([p.moves[lo:], p.moves[:lo + n - n_all]])
        r = om.eval_incremental(x, mv)
        idx, _ = O.topk(r["score"], r["flag"], TOPK)
        if idx.size:
            om.apply(x, mv[idx[0]])

    for j in range(args.warmup):
        step(j)
    t0 = time.perf_counter()
    for j in range(args.steps):
        step(args.warmup + j)
    el = time.perf_counter() - t0
    value = args.steps * n * p.S / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded lognormal Gaussian-random-field grades; no public dataset)",
            "config": {"workload": "50x50x20 blocks, S=100, T=20, 262,144 moves (50% shifts)",
                       "moves_per_step": n, "topk": TOPK},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": f"{n} moves per step (incremental FP64 evaluator + top-k + apply)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm


def batched_form(stream, flush, reps: int = K_FORM):
    """The 64-chain workload (cube sides 15..40, S in {16, 32, 64, 100}, T = 20,
    1,024..65,536 moves per chain, seeds 100..163): one persistent batched launch
    (autotuned tile, replayed from a CUDA graph) against the same 64 chains as
    sequential plain calls (mm_eval_moves + mm_topk per chain, also replayed
    from one CUDA graph).  L2 flushed before every run; times are CUDA events."""
    import torch

    import paper_2511_18296_b300 as mm
    import workloads as W

    probs = [W.chain_problem(s) for s in W.batched_chain_specs(64)]
    models = []
    for p in probs:
        m = mm.Model.from_problem(p, stream=stream)
        m.schedule_set(p.x0)
        models.append(m)
    mvs = [torch.as_tensor(p.moves, device=flush.device) for p in probs]
    evals = int(sum(p.moves.shape[0] * p.S for p in probs))
    b = mm.Batch(list(zip(models, mvs)), k=TOPK, stream=stream)
    tile, ctas, _ = b.autotune(reps=3)

    timer = StepTimer(stream, flush, R=reps)

    def seq():
        for m, mv, o in zip(models, mvs, b.out):
            m.eval_moves(mv, score=o["score"], feas=o["feas"], want_mean=False)
            m.topk(o["score"], o["feas"], TOPK, idx=o["idx"], top=o["top"], count=o["count"])

    def run_ms(fn):
        with torch.cuda.stream(stream):
            fn()
        stream.synchronize()
        ge = timer.graph([fn])
        timer.warm(ge)
        return timer.run(ge, reps)

    bt = run_ms(b.run)
    st = run_ms(seq)
    t_b, t_s = float(np.mean(bt)), float(np.mean(st))
    # the autotuner's evaluator shape per scenario count
    shapes = {}
    for c, p in enumerate(probs):
        team, pf = b.chain_shape(c)
        e = shapes.setdefault(f"S={p.S}", {"chains": 0, "team": set(), "prefetch": set()})
        e["chains"] += 1
        e["team"].add(team)
        e["prefetch"].add(pf)
    shapes = {k: {"chains": v["chains"], "team": sorted(v["team"]), "prefetch": sorted(v["prefetch"])}
              for k, v in sorted(shapes.items(), key=lambda kv: int(kv[0][2:]))}
    b.close()
    # each scenario class alone (same tile): where the batch's time goes
    peaks, which = measured_peaks()
    per_class = {}
    for S in sorted({p.S for p in probs}):
        sel = [c for c, p in enumerate(probs) if p.S == S]
        bc = mm.Batch([(models[c], mvs[c]) for c in sel], k=TOPK, stream=stream)
        bc.set_tile(tile, ctas)
        ct = run_ms(bc.run)
        bc.close()
        ms_c = float(np.median(ct))
        alg_c = float(sum(algorithmic_bytes(probs[c].moves, S) for c in sel))
        nm = int(sum(probs[c].moves.shape[0] for c in sel))
        per_class[f"S={S}"] = {"chains": len(sel), "moves": nm, "ms_alone": ms_c,
                               "moves_per_us": nm / (ms_c * 1e3),
                               "roofline_frac_alone": alg_c / (ms_c * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    alg = float(sum(algorithmic_bytes(p.moves, p.S) for p in probs))
    return {"workload": "64 chains: cubes of side 15..40, S in {16, 32, 64, 100}, T=20, 1,024..65,536 moves each",
            "evals_per_run": evals, "chains": 64, "launches_per_run": 1,
            "ms_per_run": t_b, "time": stats(bt), "value": evals / (t_b * 1e-3), "unit": UNIT,
            "algorithmic_bytes_per_run": alg,
            "roofline_frac": alg / (t_b * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "peak_source": f"{which} (MEASURED_PEAKS.json hbm_gbs)",
            "tile": {"moves_per_item": tile, "ctas_per_sm": ctas, "chosen_by": "mm_batch_autotune"},
            "chain_shapes": {"desc": "team width (lanes per move) and L1 prefetch distance per scenario count, "
                                     "chosen by mm_batch_autotune after the tile (kept only when > 1 % faster)",
                             "by_S": shapes},
            "per_class_alone": {"desc": "each scenario count's chains as a batch of their own, same tile: the "
                                        "per-move decode and feasibility work is the same at every S, so the "
                                        "byte rate falls with S",
                                "by_S": per_class},
            "sequential_plain": {"desc": "64 x (mm_eval_moves + mm_topk), one CUDA graph", "launches_per_run": 128,
                                 "ms_per_run": t_s, "time": stats(st), "value": evals / (t_s * 1e-3)},
            "speedup_vs_sequential": t_s / t_b}


def stress_form(stream, flush, reps: int = 20, n_accept: int = 1000):
    """The 100x100x40 = 400,000-block workload, S = 500, T = 30, 1,048,576
    moves (70 % shifts; seed 3).  Its 806 MB of value rows exceed L2, so here
    the evaluation streams them from DRAM.  Timed (CUDA events around CUDA-graph
    replays, L2 flushed before each): the plain and compensated evaluation
    launches and the search step (evaluate + top-32, then the apply launch).
    Untimed: n_accept accepted moves (compensated sums, best feasible move of
    the batch, applied on the device) beside an FP32 shadow of the running
    totals; returns the report and (problem, final schedule, FP64 NPV_s, FP32
    shadow NPV_s) for the oracle's comparison in the CPU leg."""
    import torch

    import paper_2511_18296_b300 as mm
    import workloads as W

    dev = flush.device
    p = W.config("stress_400k")
    m = mm.Model.from_problem(p, stream=stream)
    m.schedule_set(p.x0)
    mv = torch.as_tensor(p.moves, device=dev)
    n = p.moves.shape[0]
    score = torch.empty(n, dtype=torch.float32, device=dev)
    feas = torch.empty(n, dtype=torch.uint8, device=dev)
    idx = torch.empty(TOPK, dtype=torch.int32, device=dev)
    top = torch.empty(TOPK, dtype=torch.float32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)

    timer = StepTimer(stream, flush, R=reps)
    times = {}

    def time_fn(fn, name, R=None, reset=False):
        with torch.cuda.stream(stream):
            fn()
        stream.synchronize()
        ge = timer.graph([fn], R=R)
        timer.warm(ge)
        m.schedule_set(p.x0)
        times[name] = timer.run(ge, reps, between=(lambda: m.schedule_set(p.x0)) if reset else None)
        return float(np.mean(times[name]))

    plain_ms = time_fn(lambda: m.eval_moves(mv, score=score, feas=feas, want_mean=False), "eval")
    kahan_ms = time_fn(lambda: m.eval_moves(mv, score=score, feas=feas, want_mean=False, kahan=True), "kahan")
    # from the initial schedule the batch's best move improves the NPV for a
    # few steps only (then it is a no-op): graphs of 5 steps, the schedule
    # reset between replays, so that every timed step applies a move
    step_ms = time_fn(lambda: m.search_step(mv, k=TOPK, apply=True, score=score, feas=feas, idx=idx, top=top,
                                            count=cnt), "step", R=5, reset=True)
    # drift: FP64 running totals beside their FP32 shadow over n_accept applies
    m.set_fp32_shadow(True)
    m.schedule_set(p.x0)
    accepted = steps = improving = 0
    with torch.cuda.stream(stream):
        while accepted < n_accept and steps < n_accept + n_accept // 5:
            m.eval_moves(mv, score=score, feas=feas, want_mean=False, kahan=True)
            m.topk(score, feas, 1, idx=idx[:1], top=top[:1], count=cnt)
            m.apply_best(mv, idx[:1], cnt)
            accepted += m.last_apply()[0]  # a feasible no-op counts as applied
            improving += int(cnt[0].item() > 0 and top[0].item() > 0.0)
            steps += 1
    x = m.schedule_get()
    drift_in = (p, x, m.npv()[0], m.fp32_shadow_npv(), accepted, improving)
    m.close()
    alg = algorithmic_bytes(p.moves, p.S)
    peaks, which = measured_peaks()
    evals = n * p.S
    return {"workload": "100x100x40 = 400,000 blocks, S=500, T=30, 1,048,576 moves (70% shifts, 30% swaps)",
            "desc": "value rows (806 MB) larger than L2: the evaluation reads them from DRAM",
            "algorithmic_bytes_per_launch": alg,
            "eval_kernel_ms": plain_ms, "eval_time": stats(times["eval"]), "eval_roofline_frac": alg / (plain_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "eval_value": evals / (plain_ms * 1e-3),
            "compensated_eval_kernel_ms": kahan_ms, "compensated_eval_time": stats(times["kahan"]),
            "compensated_eval_roofline_frac": alg / (kahan_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "step_ms": step_ms, "step_time": stats(times["step"]), "step_desc": "mm_search_step: evaluate + top-32 + apply the best move, one launch",
            "value": evals / (step_ms * 1e-3), "unit": UNIT,
            "peak_source": f"{which} (MEASURED_PEAKS.json hbm_gbs)",
            "accepted_moves": accepted, "improving_moves": improving, "steps": steps}, drift_in


def shard_arm(args, p, world: int, rank: int, dev):
    """One batch split over the ranks (strong scaling): each step is
    dist.model_sharded_step, the fused step with apply off on the rank's
    slice, an all-gather of every rank's k keys over NCCL, the exact merge and
    the device apply of the winner on every replica.  Steps run eagerly (the
    collectives are not captured in a graph), each bracketed by CUDA events
    after an L2 flush; value = evaluations of the whole batch / max-over-ranks
    step time."""
    import torch
    import torch.distributed as dist

    import paper_2511_18296_b300 as mm
    from paper_2511_18296_b300 import dist as D

    if world == 1 and not dist.is_initialized():  # a world of one: the same calls, nothing to exchange
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            os.environ.setdefault("MASTER_PORT", str(sk.getsockname()[1]))
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=0, world_size=1, device_id=dev)
    m = mm.Model.from_problem(p)
    assert m.schedule_set(p.x0)
    moves_d = torch.as_tensor(p.moves, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    m.set_stream(stream)
    for _ in range(max(args.warmup, 3)):
        D.model_sharded_step(m, moves_d, TOPK)
    m.schedule_set(p.x0)
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_start = time.time()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            D.model_sharded_step(m, moves_d, TOPK)
            e1.record(stream)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_end = time.time()
    ts = torch.tensor([e0.elapsed_time(e1) for e0, e1 in ev], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(ts, op=dist.ReduceOp.MAX)
    ts = ts.cpu().numpy()
    n, S = p.moves.shape[0], p.S
    line = {"metric": METRIC, "value": n * S * K / (ts.sum() * 1e-3), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": float(ts.mean()), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded lognormal Gaussian-random-field grades; no public dataset)",
            "config": {"workload": "50x50x20 = 50,000 blocks, S=100, T=20, 262,144 moves (50% shifts, 50% swaps)",
                       "step": "dist.model_sharded_step: fused step on the rank's slice, all-gather of k keys, "
                               "merge, device apply of the winner on every replica",
                       "topk": TOPK, "l2": "flushed before every step (256 MB write outside the step events)",
                       "timing": "CUDA events around each eagerly launched step, max over ranks",
                       "parallelism": f"one batch sharded x{world}",
                       "exchange_bytes_per_rank_per_step": TOPK * 12 + 8},
            "step_time": stats(ts), "clocks": clk.summary(t_start, t_end),
            "gpu_launches": 3 * K}  # per step: the fused step, the merge's top-k and the apply (plus torch gathers)
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import paper_2511_18296_b300 as mm
    import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    p = W.config(WORKLOAD)
    if args.shard:
        return shard_arm(args, p, world, rank, dev)
    if rank > 0:  # weak scaling: every rank its own independent batch of moves
        rng = np.random.default_rng(np.random.SeedSequence([1, rank]))
        p.moves = W.random_moves(p.x0, p.T, p.moves.shape[0], 0.5, rng)
    n, S = p.moves.shape[0], p.S
    m = mm.Model.from_problem(p)
    assert m.schedule_set(p.x0)
    moves_d = torch.as_tensor(p.moves, device=dev)
    score = torch.empty(n, dtype=torch.float32, device=dev)
    feas = torch.empty(n, dtype=torch.uint8, device=dev)
    idx = torch.empty(TOPK, dtype=torch.int32, device=dev)
    top = torch.empty(TOPK, dtype=torch.float32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # All work runs on one stream; steps are replayed from CUDA graphs so that
    # host launch overhead never shows up as idle time inside the step events.
    stream = torch.cuda.Stream(device=dev)
    m.set_stream(stream)

    def fused():
        m.search_step(moves_d, k=TOPK, apply=True, score=score, feas=feas, idx=idx, top=top, count=cnt)

    def plain_eval():
        m.eval_moves(moves_d, score=score, feas=feas, want_mean=False)

    def plain_rest():
        m.topk(score, feas, TOPK, idx=idx, top=top, count=cnt)
        m.apply_best(moves_d, idx, cnt)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            flush.zero_()
            fused()
            plain_eval()
            plain_rest()
    stream.synchronize()

    timer = StepTimer(stream, flush, R=K_FORM)

    def form_ms(fns, K=None, reset=True):
        """Per-step device times of a form: K steps (K_FORM by default) from
        the initial schedule, after three untimed ones."""
        ge = timer.graph(fns)
        timer.warm(ge)
        if reset:
            m.schedule_set(p.x0)
        return timer.run(ge, K or K_FORM)

    K = args.steps
    g_step = timer.graph([fused], R=K if K <= 50 else 50)
    with ClockSampler(local) as clk:
        t_load = time.time()
        timer.warm(g_step, seconds=0.3)  # the clocks under load before the timed region
        m.schedule_set(p.x0)  # every timed run starts from the same schedule
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_start = time.time()
        # every 50 steps the schedule goes back to the initial one (untimed,
        # between replays): from it, the batch's best move improves the NPV for
        # about 190 steps, after which the best move is a no-op and a step
        # would apply nothing; so every timed step applies a move
        step_t = timer.run(g_step, K, between=lambda: m.schedule_set(p.x0))
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_end = time.time()
    total_ms = float(sum(step_t))
    step_avg_ms = total_ms / K
    step_stats = stats(step_t)
    applied, npv_mean, _ = m.last_apply()
    # the plain form (one launch per call) and the compensated-sum evaluator, same workload
    eval_t = form_ms([plain_eval])
    plain_eval_ms = float(np.mean(eval_t))
    plain_t = form_ms([plain_eval, plain_rest])
    plain_step_ms = float(np.mean(plain_t))
    kahan_t = form_ms([lambda: m.eval_moves(moves_d, score=score, feas=feas, want_mean=False, kahan=True)])
    kahan_eval_ms = float(np.mean(kahan_t))
    m.schedule_set(p.x0)
    # violation magnitudes of the batch (epsilon-relaxed fitness), same moves
    cap_ex = torch.empty(n, dtype=torch.int64, device=dev)
    prec_ex = torch.empty(n, dtype=torch.int32, device=dev)
    viol = lambda: m.eval_violation(moves_d, cap_ex, prec_ex)  # noqa: E731
    with torch.cuda.stream(stream):
        viol()
    viol_t = form_ms([viol], reset=False)
    viol_ms = float(np.mean(viol_t))
    # differentiated form: relaxed objective forward and adjoint on the same model
    xr = torch.as_tensor(W.relaxed_x(p.B, p.T, 2), device=dev)
    gr = torch.as_tensor(p.grade.astype(np.float32), device=dev)
    gJ = torch.ones(1, dtype=torch.float64, device=dev)
    fwd = lambda: m.relaxed_forward(xr, gr)  # noqa: E731

    def fwd_bwd():
        _, npv_r, ot_r = m.relaxed_forward(xr, gr)
        m.relaxed_backward(xr, gr, npv_r, ot_r, gJ)

    with torch.cuda.stream(stream):
        fwd_bwd()
    stream.synchronize()
    fwd_t = form_ms([fwd], reset=False)
    rel_fwd_ms = float(np.mean(fwd_t))
    both_t = form_ms([fwd_bwd], reset=False)
    rel_both_ms = float(np.mean(both_t))
    # weighted form: the same model and batch with uncertainty weights sigma(s,t)
    mw = mm.Model.from_problem(p, sigma=W.uncertainty_weights(p.T, p.S))
    mw.schedule_set(p.x0)
    mw.set_stream(stream)
    w_eval = lambda: mw.eval_moves(moves_d, score=score, feas=feas, want_mean=False)  # noqa: E731
    w_step = lambda: mw.search_step(moves_d, k=TOPK, apply=True, score=score, feas=feas, idx=idx, top=top,  # noqa: E731
                                    count=cnt)
    with torch.cuda.stream(stream):
        w_eval()
        w_step()
    stream.synchronize()
    ge = timer.graph([w_eval])
    timer.warm(ge)
    mw.schedule_set(p.x0)
    w_eval_t = timer.run(ge, K_FORM)
    w_eval_ms = float(np.mean(w_eval_t))
    ge = timer.graph([w_step])
    timer.warm(ge)
    mw.schedule_set(p.x0)
    w_step_t = timer.run(ge, K_FORM)
    w_step_ms = float(np.mean(w_step_t))
    # scores of a seeded sample of the batch at the initial schedule, for the
    # accuracy report against the FP64 oracle (made in the CPU leg)
    acc_sel = np.sort(np.random.default_rng(5).choice(n, min(n, 4096), replace=False))
    mv_acc = torch.as_tensor(p.moves[acc_sel], device=dev)
    acc_gpu = {}
    with torch.cuda.stream(stream):
        mw.schedule_set(p.x0)
        acc_gpu["weighted"] = mw.eval_moves(mv_acc, want_mean=False)
        m.schedule_set(p.x0)
        acc_gpu["plain"] = m.eval_moves(mv_acc, want_mean=False)
        acc_gpu["compensated"] = m.eval_moves(mv_acc, want_mean=False, kahan=True)
        m.schedule_set(p.x0)
        full_s, full_f, _ = m.eval_moves(moves_d, want_mean=False)
    stream.synchronize()
    acc_gpu = {k: (v[0].cpu().numpy(), v[1].cpu().numpy()) for k, v in acc_gpu.items()}
    acc_full = (full_s.cpu().numpy(), full_f.cpu().numpy())
    mw.close()

    # end to end through the public API with host buffers: every step copies
    # its batch of moves from pinned host memory and reads its result (the
    # top-k and count) back to pinned host memory.  Double-buffered, as a
    # search loop runs it: batch k+1 is copied on a copy stream while step k
    # computes, step k's result is read back on a third stream (so the
    # compute stream never waits on a transfer), and the host does not wait on
    # each step (stream order and events keep the buffers safe); the L2 flush
    # stays inside every step (on the compute stream, before the step), so it
    # is timed too.  The NPV statistics are read once, after the last step.
    K2 = max(20, min(100, K))  # within the ~190 steps in which the best move still improves the NPV
    # the batch travels in the compact 4-byte form (mm_search_step_packed
    # decodes it inside the step's launch) when the model allows it, else as
    # 8-byte moves
    packed = p.B + p.T + 1 <= 65536 and p.S <= 768
    if packed:
        moves_h = torch.from_numpy(mm.pack_moves(p.moves, p.B, p.T).view(np.int32)).pin_memory()
    else:
        moves_h = torch.from_numpy(p.moves).pin_memory()
    torch.cuda.set_stream(stream)
    # each step's outputs in one device buffer (idx, top, count), read back with one copy
    outs_d = [torch.empty(2 * TOPK + 1, dtype=torch.int32, device=dev) for _ in range(2)]
    outs_h = [torch.empty(2 * TOPK + 1, dtype=torch.int32).pin_memory() for _ in range(2)]
    bufs = [torch.empty_like(moves_h, device=dev) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    # the readback has a stream of its own: queued on the copy stream, the
    # next batch's copy would wait behind it (the next-but-one batch's copy
    # can start only once the step two back has finished)
    read_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]  # batch k is on the device
    freed = [torch.cuda.Event() for _ in range(2)]   # step k no longer reads its batch buffer
    done = [torch.cuda.Event() for _ in range(2)]    # step k's outputs are written
    read = [torch.cuda.Event() for _ in range(2)]    # step k's outputs are in host memory
    for e in freed + read:
        e.record(stream)

    def issue_copy(k):
        b = k % 2
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(freed[b])  # step k-2 is done with this buffer
            bufs[b].copy_(moves_h, non_blocking=True)
            copied[b].record(copy_stream)

    def e2e_run(steps):
        issue_copy(0)
        for k in range(steps):
            b = k % 2
            o = outs_d[b]
            flush.zero_()
            stream.wait_event(copied[b])
            stream.wait_event(read[b])  # step k-2's outputs have been read back
            step_fn = m.search_step_packed if packed else m.search_step
            step_fn(bufs[b], k=TOPK, apply=True, score=score, feas=feas, idx=o[:TOPK],
                    top=o[TOPK:2 * TOPK].view(torch.float32), count=o[2 * TOPK:])
            freed[b].record(stream)
            done[b].record(stream)
            if k + 1 < steps:
                issue_copy(k + 1)
            with torch.cuda.stream(read_stream):
                read_stream.wait_event(done[b])
                outs_h[b].copy_(o, non_blocking=True)
                read[b].record(read_stream)
        torch.cuda.synchronize()
        return m.last_apply()[1]  # NPV mean after the last step's move

    m.schedule_set(p.x0)
    e2e_run(3)
    m.schedule_set(p.x0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_mean = e2e_run(K2)
    e2e_avg = (time.perf_counter() - t0) / K2

    # precision: the FP64 running totals beside an FP32 shadow of them over
    # 1,000 device applies (untimed); the CPU leg compares both with the
    # oracle's full FP64 recomputation of the final schedule
    N_APPLY = 1000
    m.set_fp32_shadow(True)
    m.schedule_set(p.x0)
    n_improving = torch.zeros(1, dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(N_APPLY):
            m.search_step(moves_d, k=TOPK, apply=True, score=score, feas=feas, idx=idx, top=top, count=cnt)
            n_improving += ((cnt[:1] > 0) & (top[:1] > 0.0)).to(torch.int64)  # the step changed the schedule
    stream.synchronize()
    drift_gpu = (m.schedule_get(), m.npv()[0], m.fp32_shadow_npv())
    n_improving = int(n_improving.item())
    m.set_fp32_shadow(False)


    # max over ranks
    local_vals = torch.tensor([total_ms, step_avg_ms, e2e_avg, plain_step_ms, plain_eval_ms],
                              dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(local_vals, op=dist.ReduceOp.MAX)
    total_ms, step_avg_ms, e2e_avg, plain_step_ms, plain_eval_ms = [float(v) for v in local_vals.cpu()]

    evals_per_step = n * S
    value = world * evals_per_step * K / (total_ms * 1e-3)
    alg = algorithmic_bytes(p.moves, S)
    peaks, which = measured_peaks()
    achieved_gbs = alg / (plain_eval_ms * 1e-3) / 1e9
    clocks = clk.summary(t_load, t_end)
    clocks["window"] = "0.3 s of untimed steps under load, then the timed steps"
    if clocks.get("sm_mhz"):
        # time x clock separates clock effects from box effects: SM cycles per step
        clocks["step_median_kcycles"] = step_stats["median_ms"] * clocks["sm_mhz"]
        clocks["eval_median_kcycles"] = float(np.median(eval_t)) * clocks["sm_mhz"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded lognormal Gaussian-random-field grades; no public dataset)",
        "config": {"workload": "50x50x20 = 50,000 blocks, S=100, T=20, 262,144 moves (50% shifts, 50% swaps)",
                   "step": ("mm_search_step: evaluate + top-32 + apply the best move, "
                            + ("one launch" if S <= 768 else "an evaluation launch and an apply launch")
                            + ", replayed from a CUDA graph"),
                   "topk": TOPK,
                   "l2": "flushed before every step (256 MB write outside the step events)",
                   "timing": ("every step bracketed by CUDA events recorded inside a CUDA graph of (flush, step) "
                              "pairs (external event nodes; the flush outside the events); 0.3 s of untimed steps "
                              "under load first; the schedule reset to the initial one (untimed) every 50 steps, so "
                              "that every timed step applies an improving move; forms: median, best and quartiles "
                              "of 50 steps from the initial schedule"),
                   "per_rank_moves": n, "parallelism": f"independent batches x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved_gbs / peaks["hbm_gbs"], "traffic": profiled_traffic(),
                     "kernel": EVAL_KERNEL + " (mm_eval_moves: one evaluation launch per batch, timed in the plain form)",
                     "kernel_ms": plain_eval_ms,
                     "step_frac": alg / (step_avg_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                     "algorithmic_bytes_per_launch": alg, "peak_source": f"{which} (MEASURED_PEAKS.json hbm_gbs)",
                     "nominal_peak": HBM_NOMINAL_GBS, "frac_of_nominal": achieved_gbs / HBM_NOMINAL_GBS},
        "step_time": step_stats,
        "plain_form": {"desc": "mm_eval_moves, then mm_topk + mm_apply_best: one launch per call, same workload",
                       "step_time": stats(plain_t), "eval_time": stats(eval_t),
                       "value": evals_per_step * world / (plain_step_ms * 1e-3), "unit": UNIT,
                       "ms_per_step": plain_step_ms, "eval_kernel_ms": plain_eval_ms,
                       "eval_roofline_frac": achieved_gbs / peaks["hbm_gbs"], "eval_achieved_gbs": achieved_gbs},
        "precision_form": {"desc": "mm_eval_moves_ex with compensated scenario sums (MM_EVAL_KAHAN); drift: NPV from "
                                   "the FP64 running totals and from an FP32 shadow after 1,000 applies, against the "
                                   "oracle's recomputation",
                           "eval_kernel_ms": kahan_eval_ms, "eval_time": stats(kahan_t),
                           "eval_roofline_frac": alg / (kahan_eval_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]},
        "weighted_form": {"desc": "uncertainty weights sigma(s,t) of Eq. 12 (synthetic, seed 4) on the same model and "
                                  "batch: evaluation launch, and the fused step (evaluate + top-32 + apply, one "
                                  "launch)",
                          "eval_kernel_ms": w_eval_ms, "eval_time": stats(w_eval_t), "step_time": stats(w_step_t),
                          "eval_roofline_frac": alg / (w_eval_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                          "step_ms": w_step_ms,
                          "value": n * p.S / (w_step_ms * 1e-3), "unit": UNIT},
        "violation_form": {"desc": "mm_eval_violation: capacity and precedence excess of every move (exact integers)",
                           "ms_per_batch": viol_ms, "moves_per_s": n / (viol_ms * 1e-3), "time": stats(viol_t)},
        "differentiated_form": {
            "desc": "relaxed objective on the same model, x[b,t] ~ Dirichlet(1) (seed 2): forward, and forward + "
                    "adjoint (dJ/dx, dJ/dg)",
            "forward_ms": rel_fwd_ms, "forward_backward_ms": rel_both_ms,
            "forward_time": stats(fwd_t), "forward_backward_time": stats(both_t),
            "algorithmic_bytes": {"forward": 4 * p.B * (p.T + p.S), "forward_backward": 4 * p.B * 3 * (p.T + p.S)},
            "forward_gbs": 4 * p.B * (p.T + p.S) / (rel_fwd_ms * 1e-3) / 1e9,
            "forward_backward_gbs": 4 * p.B * 3 * (p.T + p.S) / (rel_both_ms * 1e-3) / 1e9,
            "forward_hbm_frac": 4 * p.B * (p.T + p.S) / (rel_fwd_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "forward_backward_hbm_frac": 4 * p.B * 3 * (p.T + p.S) / (rel_both_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
            # the contractions run on the tensor cores as TF32 products with
            # hi/lo splits (O two products, V three, the adjoint's sum over
            # scenarios two): algorithmic FLOPs 2 B T S per product of the
            # definition, against the TF32 peak (the measured bf16 burst x the
            # nominal TF32 / bf16 ratio 1.1 / 2.25)
            "tensor_roofline": {
                "bound": "tensor", "unit": "TFLOP/s", "peak": peaks["bf16_tflops"] * 1.1 / 2.25,
                "peak_source": f"{which}: MEASURED_PEAKS.json bf16_tflops x nominal TF32/bf16 ratio 1.1/2.25",
                "forward_flop": 4.0 * p.B * p.T * p.S,
                "forward_backward_flop": 6.0 * p.B * p.T * p.S,
                "forward_mma_flop_with_splits": 10.0 * p.B * p.T * p.S,
                "forward_achieved": 4.0 * p.B * p.T * p.S / (rel_fwd_ms * 1e-3) / 1e12,
                "forward_frac": 4.0 * p.B * p.T * p.S / (rel_fwd_ms * 1e-3) / 1e12
                / (peaks["bf16_tflops"] * 1.1 / 2.25),
                "forward_backward_achieved": 6.0 * p.B * p.T * p.S / (rel_both_ms * 1e-3) / 1e12,
                "forward_backward_frac": 6.0 * p.B * p.T * p.S / (rel_both_ms * 1e-3) / 1e12
                / (peaks["bf16_tflops"] * 1.1 / 2.25)},
            "vs_plain_eval": {"plain_eval_ms": plain_eval_ms}},
        "e2e": {"value": evals_per_step * world / e2e_avg, "unit": UNIT,
                "h2d_bytes_per_step": int(moves_h.numel()) * moves_h.element_size(),
                "d2h_bytes_per_step": int(outs_h[0].numel()) * 4,
                "ms_per_step": e2e_avg * 1e3,
                "path": (("pinned host moves in the compact 4-byte form -> mm_search_step_packed (decoded inside "
                          "the step's launch; apply on device)" if packed else
                          "pinned host moves -> mm_search_step (apply on device)")
                         + " -> top-k and count to pinned host memory every step; "
                         "double-buffered (batch k+1 copied on a copy stream and step k-1's result read back on a third "
                         "stream while step k runs), the host not waiting on each step; L2 flush inside each step; NPV statistics "
                         "read after the last step")},
        "gpu_launches": (1 if S <= 768 else 2) * K,  # per step: the evaluation launch (top-k and apply inside when S <= 768)
        "clocks": clocks,
        "check": {"last_apply": applied, "npv_mean": npv_mean, "e2e_npv_mean": e2e_mean},
    }
    if rank == 0 and not args.no_batched:
        line["batched_form"] = batched_form(stream, flush)
    stress_in = None
    if rank == 0 and not args.no_stress:
        line["stress_form"], stress_in = stress_form(stream, flush)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, budget_s=args.cpu_budget)
        line["accuracy"] = accuracy_report(p, acc_sel, acc_gpu)
        line["accuracy"]["full_batch_plain"] = full_batch_accuracy(p, *acc_full)
        line["precision_form"]["drift"] = drift_report(p, *drift_gpu, n_apply=N_APPLY)
        line["precision_form"]["drift"]["improving_moves"] = n_improving
        if stress_in is not None:
            ps, xs, n64, n32, acc, imp = stress_in
            line["stress_form"]["drift"] = drift_report(
                ps, xs, n64, n32, n_apply=acc,
                workload="the 400,000-block model: accepted moves (compensated sums, best feasible move of the "
                         "batch) applied on the device from the initial schedule")
            line["stress_form"]["drift"]["improving_moves"] = imp
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def profile_run(form: str) -> int:
    """A short fixed launch sequence of one form for an ncu capture (no timing,
    no JSON line): four launches of the form's kernels on the 50k workload
    (the 64-chain workload for `batched`), the L2 flushed before each, so
    `-s 3 -c 1` on the form's kernel captures the fourth, cold like a bench
    step.  eval: mm_eval_moves; step: mm_search_step with apply; relaxed: the
    forward and the adjoint on its outputs; batched: mm_batch_run with 1,024
    moves per item and the maximum CTAs per SM (the autotuner's choice there)."""
    import torch

    import paper_2511_18296_b300 as mm
    import workloads as W

    dev = torch.device("cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if form == "batched":
        probs = [W.chain_problem(s) for s in W.batched_chain_specs(64)]
        models = []
        for p in probs:
            m = mm.Model.from_problem(p)
            m.schedule_set(p.x0)
            models.append(m)
        mvs = [torch.as_tensor(p.moves, device=dev) for p in probs]
        b = mm.Batch(list(zip(models, mvs)), k=TOPK)
        b.set_tile(1024, 0)  # the tile the autotuner picks on this workload
        run = b.run
    else:
        p = W.config(WORKLOAD)
        m = mm.Model.from_problem(p)
        m.schedule_set(p.x0)
        mv = torch.as_tensor(p.moves, device=dev)
        n = mv.shape[0]
        score = torch.empty(n, dtype=torch.float32, device=dev)
        feas = torch.empty(n, dtype=torch.uint8, device=dev)
        if form == "eval":
            def run():
                m.eval_moves(mv, score=score, feas=feas, want_mean=False)
        elif form == "step":
            def run():
                m.search_step(mv, k=TOPK, apply=True, score=score, feas=feas)
        elif form == "relaxed":
            xr = torch.as_tensor(W.relaxed_x(p.B, p.T, 2), device=dev)
            gr = torch.as_tensor(p.grade.astype(np.float32), device=dev)
            gJ = torch.ones(1, dtype=torch.float64, device=dev)

            def run():
                _, npv_r, ot_r = m.relaxed_forward(xr, gr)
                m.relaxed_backward(xr, gr, npv_r, ot_r, gJ)
        else:
            raise SystemExit(f"--profile: unknown form {form!r}")
    torch.cuda.synchronize()
    for _ in range(4):
        flush.zero_()
        run()
    torch.cuda.synchronize()
    print(f"profile {form}: 4 runs done", flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-chain batched comparison")
    ap.add_argument("--no-stress", action="store_true",
                    help="skip the 400,000-block, 500-scenario DRAM-bound form (about a minute to generate)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: one batch split over the ranks, the ranks' top k exchanged and the winner "
                         "applied on every replica (strong scaling); default: an independent batch per rank")
    ap.add_argument("--profile", default=None, choices=["eval", "step", "relaxed", "batched"],
                    help="run a short fixed launch sequence of one form for an ncu capture and exit (no timing)")
    args = ap.parse_args(argv)
    if args.profile:
        return profile_run(args.profile)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
