/*
 * mm.h - C ABI of the B300 move-evaluation engine for stochastic open-pit
 * mine scheduling.
 *
 * The engine evaluates batches of candidate schedule moves (single-block
 * period shifts and block-pair swaps) against S geological grade scenarios.
 * Problem statement: Section 5.6 of the paper, Eq. 14 (objective: discounted
 * mining cost plus scenario-averaged processing value), Eq. 15 (a block is
 * mined no earlier than its direct predecessors), Eq. 16 (mined tonnage per
 * period within capacity M_t), with the second stage (Eq. 17-21) read as a
 * single processing mode: a block is ore in a scenario when processing beats
 * dumping it (Eq. 18, zero processed mass = waste), and the mill's ore tonnage
 * per period is held to a target Q_t by piecewise-linear shortfall/excess
 * penalties.  Cash flows and penalties are discounted per period by
 * d_t = (1 + r)^-t, t = 0..T-1 (Algorithm 5; Section 7.1.2).  The candidate
 * moves are those of Algorithms 4-5 (assign block b* to period t*).
 *
 * Conventions for every call:
 *   - Pointers named *_dev are device pointers owned by the caller; *_host are
 *     host pointers owned by the caller.  The library owns all model state on
 *     the device and frees it in mm_model_destroy.
 *   - Asynchronous calls (mm_eval_*, mm_topk, mm_apply_best) only enqueue work
 *     on the model's stream and return MM_OK unless an argument is invalid or a
 *     launch fails.  Synchronising calls (mm_schedule_set/get, mm_apply_move,
 *     mm_npv, mm_get_*) wait for the stream.
 *   - A bad move inside a batch (block id or period out of range) does not fail
 *     the batch: its flag is 0, its score -INFINITY, and the next synchronising
 *     call returns MM_ERR_BAD_MOVE once (sticky bit, then cleared).
 *   - Errors: every call returns an mm_status; mm_last_error() gives a message
 *     for the last failing call on the calling thread.  No call aborts, traps or
 *     falls back to the CPU.
 *   - A model is not thread-safe: one host thread at a time.
 *
 * Limits: 1 <= T <= 254 (period byte; value T means "unmined"), 1 <= S <= 1024,
 * B < 2^31, total block mass < 2^62 t, top-k k <= 1024.
 */
#ifndef MM_H
#define MM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MM_OK = 0,
    MM_ERR_INVALID_ARG = 1, /* a NULL pointer, size or value out of range */
    MM_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    MM_ERR_OOM = 3,         /* device allocation failed or over the model's memory cap */
    MM_ERR_OVERFLOW = 4,    /* tonnage sums would overflow 2^62 */
    MM_ERR_INFEASIBLE = 5,  /* mm_apply_move: the move's feasibility flag is 0; nothing changed */
    MM_ERR_BAD_MOVE = 6,    /* a move referenced a block or period out of range */
    MM_ERR_TIMEOUT = 7,     /* a bounded device wait ran out */
    MM_ERR_STATE = 8        /* call out of order (e.g. eval before mm_schedule_set) */
} mm_status;

/* Opaque model: block model, scenarios, schedule and derived device state. */
typedef struct mm_model mm_model;

/* One candidate move (8 bytes; arrays of moves are [n] of these).
 *   arg >= 0 : swap the periods of blocks b1 and arg;
 *   arg <  0 : shift block b1 to period -arg-1 (0..T; T = leave unmined).
 * A shift to the block's own period, a swap of a block with itself or of two
 * blocks in the same period changes nothing (delta 0). */
typedef struct {
    int32_t b1;
    int32_t arg;
} mm_move;

/* Model description (Section 5.6 parameter table: blocks, n_s scenarios,
 * n_T periods, m_b, M_t, direct predecessors; economics of Eq. 14/17). */
typedef struct {
    int32_t n_blocks, n_scenarios, n_periods; /* B, S, T */
    /* Precedence: either a grid for the 1-5 pattern (nx*ny*nz == B, block
     * b = x + nx*(y + ny*z), z = 0 on top; the predecessors of (x,y,z) are
     * (x,y,z-1), (x+-1,y,z-1), (x,y+-1,z-1), clipped at the boundary), or
     * nx = ny = nz = 0 and a CSR of direct predecessors (host arrays,
     * pred_ptr[B+1], pred_idx[pred_ptr[B]]; must describe a DAG). */
    int32_t nx, ny, nz;
    const int32_t *pred_ptr, *pred_idx;
    const uint32_t *mass_t;         /* [B] host, block mass m_b in tonnes, > 0 */
    const double *grade;            /* [B][S] host, g/t, scenario fastest, finite, >= 0 */
    const uint64_t *cap_t;          /* [T] host, mining capacity M_t in tonnes */
    const uint64_t *mill_target_t;  /* [T] host, mill ore target Q_t in tonnes */
    double price, recovery;         /* $/g, recovered fraction */
    double mining_cost, proc_cost;  /* $/t mined, $/t processed */
    double shortfall_pen, excess_pen; /* $/t below / above Q_t */
    double discount_rate;           /* r, per period */
    double lambda;                  /* risk weight of score = mean - lambda*std */
    /* Optional uncertainty weights sigma(s,t) of Section 5.6 (Eq. 12:
     * ENPV_{b,s,t} = sigma(s,t) (Revenue - ProcessingCost)): [T][S] host,
     * period-major, finite, >= 0, or NULL for none.  They scale the processing
     * margin m((g*price)*recovery - pc) of a block that is ore in scenario s
     * and mined in period t; the mining cost m*mc and the mill penalties are
     * not weighted.  See mm_model_create for what changes with them. */
    const double *sigma;
    void *cuda_stream;              /* cudaStream_t for all work (NULL = default stream) */
} mm_model_desc;

/* Create a model: copies the inputs to the device, classifies every
 * (block, scenario) as ore or waste in FP64 with the rule
 * (g*price)*recovery > proc_cost (strict), and builds the FP32 per-block
 * value rows v[b][s] = ore ? m((g*price)*recovery - pc) - m*mc : -m*mc and the
 * ore bitmask.  The model has no schedule yet.  Synchronising.
 * With uncertainty weights (desc->sigma) the rows hold the ore margin
 * ore ? m((g*price)*recovery - pc) : 0, every NPV is
 *   NPV_s = sum_t d_t (sigma(s,t) margin_t,s - mc mined_t - pen_t(ore_t,s)),
 * the evaluator reads a [T+1][T+1][S_pad] FP32 table of the weighted discount
 * differences sigma(s,b) d_b - sigma(s,a) d_a, mm_search_step is one launch
 * when the weighted fast form applies (equal masses, S % 4 == 0) and runs as the
 * separate evaluation, top-k and apply launches otherwise, and the relaxed
 * objective and the batched evaluator refuse the model (MM_ERR_INVALID_ARG).
 * Errors: MM_ERR_INVALID_ARG (NULL, sizes, non-finite or negative grade or
 * weight, zero mass, bad CSR), MM_ERR_OVERFLOW, MM_ERR_OOM, MM_ERR_CUDA. */
mm_status mm_model_create(const mm_model_desc *desc, mm_model **out);

/* Free all device state of the model.  NULL is ignored. */
void mm_model_destroy(mm_model *m);

/* Use another stream for subsequent calls (NULL = default stream). */
mm_status mm_set_stream(mm_model *m, void *cuda_stream);

/* Install a schedule: period_host[B] in 0..T (T = unmined).  Rebuilds, from
 * scratch, the per-period mined tonnage, per-(period, scenario) ore tonnage
 * (int64, exact), metal (FP64), the per-scenario NPV (FP64) and the tables the
 * move evaluator reads; this also discards any drift accumulated by applies.
 * *base_feasible_out (nullable) receives 1 when the schedule satisfies Eq. 15
 * on every arc and Eq. 16 in every period.  Synchronising. */
mm_status mm_schedule_set(mm_model *m, const uint8_t *period_host, int *base_feasible_out);

/* Copy the current schedule to period_host[B].  Synchronising. */
mm_status mm_schedule_get(mm_model *m, uint8_t *period_host);

/* Evaluate n moves against the current schedule (Algorithm 5's candidate
 * evaluation, per scenario).  For move i and scenario s:
 *   delta_s  = NPV_s(x') - NPV_s(x)  (value change plus discounted change of
 *              the mill-deviation penalties of the affected periods);
 *   score[i] = mean_s delta_s - lambda * std_s delta_s (population std);
 *   feasible[i] = 1 iff every precedence arc with an end in a moved block holds
 *              in x' and every period a moved block leaves or enters is within
 *              capacity in x' (exact integer test; equals full feasibility of x'
 *              when x is feasible);
 *   mean[i]  = mean_s delta_s (mean_dev may be NULL).
 * moves_dev[n] (8-byte aligned), score_dev[n], feasible_dev[n], mean_dev[n]:
 * device memory.  n = 0 is allowed.  Asynchronous. */
mm_status mm_eval_moves(mm_model *m, const mm_move *moves_dev, int64_t n, float *score_dev,
                        uint8_t *feasible_dev, float *mean_dev);

/* Compact 4-byte moves, for moving candidate batches from host memory at half
 * the bytes (the paper has no counterpart; its moves are generated where they
 * are evaluated).  Packed move p = (b1 << 16) | code with b1 < 2^16 and
 *   code < B          : swap b1 with block `code`   -> mm_move {b1, code};
 *   code = 65535 - t  : shift b1 to period t, 0 <= t <= T (T = leave unmined)
 *                                                   -> mm_move {b1, -t - 1};
 * usable when B + T + 1 <= 65536 (MM_ERR_INVALID_ARG otherwise).  Codes between
 * B and 65535 - T, and b1 >= B, decode to a bad move {-1, -1}, which the
 * evaluator flags as such.  packed_dev[n] (4-byte aligned) and moves_dev[n]
 * (8-byte aligned): device memory; n = 0 is allowed.  Asynchronous. */
mm_status mm_unpack_moves(mm_model *m, const uint32_t *packed_dev, int64_t n, mm_move *moves_dev);

/* Violation magnitudes of n moves against the current schedule, for the
 * epsilon-relaxed fitness of the paper's search (Algorithm 2: fitness =
 * NPV - penalty max(0, violation - epsilon); Section 6, Phase 2).  The paper
 * does not define violation(S) further; this library reports, exactly:
 *   cap_excess[i]  = sum over the distinct periods t < T that a moved block
 *                    leaves or enters of max(0, mined'_t - M_t), tonnes (Eq. 16);
 *   prec_excess[i] = sum over the moved blocks b of max(0, L_b - x'_b) +
 *                    max(0, x'_b - H_b), periods, with L_b / H_b the latest
 *                    predecessor / earliest successor period in x' (0 / T when
 *                    there are none) (Eq. 15).
 * Both are 0 exactly when mm_eval_moves gives the move flag 1.  A bad move gets
 * -1 in both and raises the sticky MM_ERR_BAD_MOVE.  moves_dev[n], outputs
 * cap_excess_dev[n] (int64) and prec_excess_dev[n] (int32): device memory.
 * Asynchronous. */
mm_status mm_eval_violation(mm_model *m, const mm_move *moves_dev, int64_t n, int64_t *cap_excess_dev,
                            int32_t *prec_excess_dev);

/* Tile shape of the move evaluator (chosen by the autotuner or by hand):
 * team = lanes that evaluate one move (4, 8, 16 or 32; 0 = built-in choice),
 * ctas_per_sm = resident CTAs per SM of the persistent grid (0 = occupancy
 * maximum), stages = how block rows reach the lanes: 0 = direct global loads,
 * 1..4 = bulk copies into shared memory with that many batches in flight per
 * warp, -1 = built-in choice; prefetch = with direct loads, how many batches
 * ahead the rows are prefetched into L1 (0..8, -1 = built-in choice: 0 while the
 * value rows fit in L2, 1 when they are larger and come from DRAM).  team must
 * leave at most 8 scenario quads per lane (ceil(ceil(S/4)/team) <= 8), else
 * MM_ERR_INVALID_ARG. */
mm_status mm_set_tile(mm_model *m, int32_t team, int32_t ctas_per_sm, int32_t stages, int32_t prefetch);

/* Evaluation options for mm_eval_moves_ex. */
enum {
    MM_EVAL_PLAIN = 0,     /* FP32 scenario sums, tree reduction */
    MM_EVAL_KAHAN = 1,     /* compensated scenario sums: the mean's sum by Kahan's update per
                              scenario quad (the quad's four deltas summed first; error-free
                              TwoSum merges across the lanes of a team), the variance by the
                              corrected two-pass formula: the sum of squared deviations minus
                              (sum of deviations)^2 / S, which removes the error of the rounded
                              mean, with the deviations' sum formed as the compensated total
                              minus S times the mean (the squares need no compensation: they
                              are non-negative, nothing cancels) */
    MM_EVAL_GENERIC = 2    /* use the evaluator whose scenario loop is shaped at run time even
                              where a compile-time-shaped one exists (same results; for
                              cross-checking the two) */
};

/* mm_eval_moves with options and an optional per-scenario output:
 * delta_dev[n][S] (FP32, row i = move i; may be NULL). */
mm_status mm_eval_moves_ex(mm_model *m, const mm_move *moves_dev, int64_t n, float *score_dev,
                           uint8_t *feasible_dev, float *mean_dev, float *delta_dev, int32_t options);

/* The k feasible moves with the largest score, ties to the lower move index
 * (replaces the paper's atomic per-CTA best-move reduction, Algorithm 5 and
 * Section 6 Phase 5, with an exact, deterministic selection).  Reads
 * score_dev[n], feasible_dev[n]; writes idx_dev[k] (move indices, best first),
 * topscore_dev[k] and *count_dev = min(k, number of feasible moves with a
 * non-NaN score); topscore_dev[j] = score_dev[idx_dev[j]], except that a
 * -0.0 score may come back as +0.0 (-0.0 and +0.0 compare equal in the
 * selection).  1 <= k <= 1024.
 * Device memory; asynchronous.  k <= 32: one launch; per-CTA warp lists of the
 * 32 best keys, merged in two levels by the CTAs that finish last (model-owned
 * lists, no allocation).  k > 32: histogram cut plus radix select in
 * model-owned scratch, grown on demand (the first call with a larger n
 * allocates).  Both give the same, exact result. */
mm_status mm_topk(mm_model *m, const float *score_dev, const uint8_t *feasible_dev, int64_t n,
                  int32_t k, int32_t *idx_dev, float *topscore_dev, int32_t *count_dev);

/* One local-search step, one launch for S <= 768 (Algorithm 4's evaluate-then-assign
 * loop body with Algorithm 5's candidate evaluation): evaluates the n moves
 * exactly as mm_eval_moves (score_dev[n], feasible_dev[n]), selects the k best
 * feasible ones exactly as mm_topk (idx_dev[k], topscore_dev[k], *count_dev;
 * 1 <= k <= 32), and, if apply != 0, applies the best one on the device exactly
 * as mm_apply_best (outcome via mm_last_apply).  The launch runs one CTA of
 * 768 threads per SM (mm_set_tile's ctas_per_sm does not apply to it); each
 * warp keeps its 32 best keys in registers (warp shuffles), each CTA merges
 * its warps' lists and publishes one list, and the CTA that finishes last
 * (a ticket, no waiting) ranks the lists' heads, selects the 32 best keys
 * from the lists that can hold one of them and writes the top k.  When S <= 768 that
 * final CTA also applies the best move from the record the evaluation kept of
 * it (its blocks and periods): the tonnage, schedule words and penalty tables
 * (everything the next evaluation reads) in this launch, the move's FP64
 * totals (metal, net cash per period, NPV_s) by the next step's CTAs on this
 * model (a share of the scenarios each, while they still evaluate) or, before
 * that, by the library ahead of any call that reads or changes those totals
 * (mm_npv, mm_last_apply, mm_get_metal, mm_apply_move, mm_apply_best,
 * mm_get_fp32_shadow_npv, mm_set_fp32_shadow, mm_batch_run with apply);
 * mm_schedule_set discards it.  Every total is the same bits as with
 * mm_apply_best.  Above 768 scenarios a one-CTA apply launch follows.  Needs
 * equal block masses (else MM_ERR_INVALID_ARG; use the separate calls).
 * Calls on one model must not overlap on the GPU (they share the model's
 * list storage).  Asynchronous. */
mm_status mm_search_step(mm_model *m, const mm_move *moves_dev, int64_t n, int32_t k, int32_t apply,
                         float *score_dev, uint8_t *feasible_dev, int32_t *idx_dev, float *topscore_dev,
                         int32_t *count_dev);

/* mm_search_step on a batch in the compact 4-byte form of mm_unpack_moves,
 * decoded inside the evaluation launch (no unpack launch, half the bytes of
 * moves read): packed_dev[n] (device memory, 4-byte aligned; NULL allowed
 * when n = 0).  Every output, the applied move and the sticky status are
 * exactly those of mm_unpack_moves followed by mm_search_step on the same
 * batch; codes that name no move are bad moves (feasible = 0, score = -inf,
 * sticky MM_ERR_BAD_MOVE).  Only where the whole step is one launch: needs
 * B + T + 1 <= 65536, equal block masses, S <= 768 when apply != 0, and, with
 * uncertainty weights, the weighted fast form (S % 4 == 0); otherwise
 * MM_ERR_INVALID_ARG (use mm_unpack_moves and mm_search_step).
 * Asynchronous. */
mm_status mm_search_step_packed(mm_model *m, const uint32_t *packed_dev, int64_t n, int32_t k, int32_t apply,
                                float *score_dev, uint8_t *feasible_dev, int32_t *idx_dev, float *topscore_dev,
                                int32_t *count_dev);

/* Timing hook; the paper has no counterpart.  When cuda_event (a cudaEvent_t
 * created with timing enabled, owned by the caller) is not NULL, every later
 * mm_search_step records it on the model's stream between its evaluation launch
 * (which includes the top-k selection) and its apply launch, so that the two
 * can be timed apart; while the stream
 * is being captured into a CUDA graph the record becomes an external event node.
 * NULL turns the hook off.  A failed record is MM_ERR_CUDA. */
mm_status mm_set_step_event(mm_model *m, void *cuda_event);

/* ---- Batched multi-chain evaluation (many search chains, one launch) ----
 *
 * The paper's search runs a population of independent chains (Table 3: a
 * population of 100; Section 6's candidate chunks).  A batch evaluates one
 * move batch per chain -- chains with different block models, scenario counts
 * and batch sizes -- in ONE persistent launch fed by a device work queue of
 * (chain, move range) items, each chain's result exactly what mm_search_step
 * gives for that chain alone (scores, flags, top k; the best move applied when
 * apply != 0; the chain runs with the team width the single-model path picks
 * by default, whatever mm_set_tile says).
 *
 * A chain names its model (schedule installed, equal block masses, T <= 64;
 * S <= 256 when applying; no two chains share a model) and the caller's device
 * buffers: moves_dev[n_moves], score_dev[n_moves], feasible_dev[n_moves],
 * idx_dev[k], topscore_dev[k], count_dev[1].  The buffers are fixed at
 * creation; a caller changes a chain's moves by rewriting moves_dev (n_moves is
 * fixed).  The batch owns its queue and list storage (allocated at creation and
 * on a tile change).  mm_batch_run is asynchronous on cuda_stream, allocates
 * nothing and never synchronises, so it can be captured into a CUDA graph;
 * work on the chains' own model streams must be ordered before it by the
 * caller.  Bad moves: feasible = 0 and the chain's model raises its sticky
 * MM_ERR_BAD_MOVE.  There are no device-side waits (each chain is finished by
 * the CTA that completes its last item, by ticket). */
typedef struct {
    mm_model *model;
    const mm_move *moves_dev;
    int64_t n_moves;
    float *score_dev;
    uint8_t *feasible_dev;
    int32_t *idx_dev;
    float *topscore_dev;
    int32_t *count_dev;
} mm_chain;

typedef struct mm_batch mm_batch;

/* 1 <= k <= 32.  MM_ERR_INVALID_ARG / MM_ERR_STATE on a chain that breaks the
 * rules above (the message names the chain), MM_ERR_CUDA on allocation. */
mm_status mm_batch_create(const mm_chain *chains, int32_t n_chains, int32_t k, int32_t apply,
                          void *cuda_stream, mm_batch **out);
void      mm_batch_destroy(mm_batch *b);

/* One evaluation of every chain (plus the applies): asynchronous. */
mm_status mm_batch_run(mm_batch *b);

/* Tile shape: moves per queue item (a multiple of 64) and resident CTAs per SM
 * of the persistent grid (0 = the occupancy maximum).  Rebuilds the queue
 * (synchronous; not while a run or a graph replay is in flight). */
mm_status mm_batch_set_tile(mm_batch *b, int32_t moves_per_item, int32_t ctas_per_sm);
mm_status mm_batch_get_tile(const mm_batch *b, int32_t *moves_per_item, int32_t *ctas_per_sm,
                            int32_t *n_items);

/* Evaluator shape of one chain: team width (lanes per move: 4, 8, 16 or 32,
 * with at most 4 scenario quads per lane, 8 for 32-lane teams; 0 = the
 * single-model default) and L1 prefetch distance in evaluation batches (0..8;
 * -1 = none).  With the default team a chain's results are the bits of the
 * single-model path; another team width adds the scenario sums in another
 * order (the same tolerance against the FP64 oracle).  Synchronous (uploads
 * the chain's descriptor); not while a run or a graph replay is in flight.
 * MM_ERR_INVALID_ARG on a chain index, team width or distance out of range. */
mm_status mm_batch_set_chain(mm_batch *b, int32_t chain, int32_t team, int32_t prefetch);
mm_status mm_batch_get_chain(const mm_batch *b, int32_t chain, int32_t *team, int32_t *prefetch);

/* Autotuner, in three passes, each timing `reps` runs (after a warm-up run)
 * with CUDA events on the batch's stream: (1) every tile shape (moves per item
 * 512 .. 16384 x CTAs per SM {max, max - 1}), keeping the fastest; (2) for
 * each scenario count among the chains, every other team width that fits
 * (mm_batch_set_chain), kept only when more than 1 % faster than the best so
 * far; (3) for each scenario count, L1 prefetch distances 0..2 for its
 * chains, kept the same way.  Returns the tile and the best mean time
 * (outputs may be NULL); the chosen team widths and distances are read with
 * mm_batch_get_chain.  Synchronous;
 * only for batches created with apply = 0 (MM_ERR_STATE otherwise), since it
 * runs the batch many times. */
mm_status mm_batch_autotune(mm_batch *b, int32_t reps, int32_t *moves_per_item, int32_t *ctas_per_sm,
                            float *best_ms);

/* mm_topk for callers that must not allocate device memory, such as code
 * that owns a fixed memory budget or pool and must not grow it, or a loop that
 * must never block the device the way cudaMalloc and cudaFree can.  The paper
 * has no counterpart: it is an interface convenience of this library.  It
 * needs no model: it selects, from score_dev[n] / feasible_dev[n], the k
 * feasible moves with the largest score exactly as mm_topk does (same outputs,
 * ties to the lower index) and enqueues the work on cuda_stream (NULL = default
 * stream).
 * Scratch: one fixed device array inside this library (about 8 MiB).  It is
 * created on a device when the library's top-k module is loaded there: when
 * the context is created under eager module loading, or at the first use of
 * the module on that device under lazy loading (the CUDA default), which may
 * be this entry point's first call; that load allocates, so make the first call
 * on a device before any fixed memory budget applies.  From then on the array
 * stays until the process exits; n must be at most 1,048,576 (else
 * MM_ERR_INVALID_ARG) and 1 <= k <= 1024.  No later call allocates: each clears
 * the parts of the array that must start at zero with an asynchronous memset
 * on cuda_stream.  The first call on a device also looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it; make
 * that first call before any stream capture.  The kept address is not valid
 * across cudaDeviceReset or a destroyed and re-created primary context in the
 * same process.  All calls share the one array, so two calls that may run at
 * the same time on the GPU (different streams, or the same device from two
 * threads) race: serialise them.  Asynchronous. */
mm_status mm_topk_noalloc(const float *score_dev, const uint8_t *feasible_dev, int64_t n, int32_t k,
                          int32_t *idx_dev, float *topscore_dev, int32_t *count_dev, void *cuda_stream);

/* Apply one move (Algorithm 4: assign S[b*] <- t*) if its feasibility flag is
 * 1: updates the schedule, the integer tonnages, the FP64 metal accumulators,
 * the per-scenario NPV and the evaluator's tables for the affected periods.
 * Returns the new NPV mean and std over scenarios (FP64; pointers nullable).
 * MM_ERR_INFEASIBLE or MM_ERR_BAD_MOVE: nothing changed.  Synchronising. */
mm_status mm_apply_move(mm_model *m, mm_move move, double *npv_mean_out, double *npv_std_out);

/* Device-side apply of the best move of a batch, for search loops that never
 * leave the GPU: if *count_dev > 0, applies moves_dev[idx_dev[0]] exactly as
 * mm_apply_move does (re-checking feasibility on the device).  The outcome
 * (applied 0/1) is kept on the device and returned by the next mm_last_apply
 * call.  moves_dev[n] is the batch idx_dev indexes (NULL allowed when n = 0); an
 * index outside 0..n-1 is treated as a bad move (nothing applied, sticky
 * MM_ERR_BAD_MOVE).  Asynchronous. */
mm_status mm_apply_best(mm_model *m, const mm_move *moves_dev, int64_t n, const int32_t *idx_dev,
                        const int32_t *count_dev);

/* Outcome of the last device-side apply (mm_apply_best, mm_search_step,
 * mm_batch_run): *applied (1 if a move was applied), and the NPV mean and
 * population std over scenarios of the model's current schedule, formed from
 * the FP64 NPV_s by this call (the search step itself does not spend time on
 * them).  Pointers nullable.  Synchronising. */
mm_status mm_last_apply(mm_model *m, int32_t *applied, double *npv_mean_out, double *npv_std_out);

/* Per-scenario NPV of the current schedule (FP64, [S], nullable) and its mean
 * and population std (nullable).  Synchronising. */
mm_status mm_npv(mm_model *m, double *npv_per_scenario_host, double *mean, double *std);

/* Sizes: any pointer may be NULL.  s_pad = row stride, in 4-byte words, of the
 * per-block device rows (S FP32 values, then the ore words; a multiple of 8). */
mm_status mm_model_info(const mm_model *m, int32_t *B, int32_t *S, int32_t *T, int32_t *s_pad);

/* Inspection (synchronising; host outputs):
 *   ore_host[B][ceil(S/32)]  bit (s % 32) of word s / 32 = ore flag of (b, s);
 *   value_host[B][S]         FP32 value rows;
 *   mined_host[T], ore_t_host[T][S]  integer tonnages of the current schedule;
 *   metal_host[T][S]         FP64 metal accumulators (grams in situ of ore). */
mm_status mm_get_ore(mm_model *m, uint32_t *ore_host);
mm_status mm_get_values(mm_model *m, float *value_host);
mm_status mm_get_tonnage(mm_model *m, int64_t *mined_host, int64_t *ore_t_host);
mm_status mm_get_metal(mm_model *m, double *metal_host);

/* ---- Relaxed objective and its adjoint (differentiable form) ----
 *
 * Eq. 14 with the extraction decision relaxed to x[b][t] in [0, 1] (row sums
 * are not forced) and the mill penalty smoothed, under the risk term
 * J = mean_s NPV_s - lambda std_s NPV_s (population std):
 *   O[t][s] = sum_b x[b][t] m_b ore[b][s],  V[t][s] = sum_b x[b][t] v[b][s],
 *   NPV_s   = sum_t d_t (V[t][s] - P_t(O[t][s])),
 *   P_t(O)  = a m_ref sp((Q_t - O) / m_ref) + e m_ref sp((O - Q_t) / m_ref),
 *   sp(z)   = log(1 + exp(beta z)) / beta
 * with d_t, Q_t, a, e, lambda and the economics of the model.  ore and v are
 * recomputed from the grades: g_dev[B][S] (FP32, device) when given, else the
 * model's own FP64 grades; the ore decision is (g * price) * recovery >
 * proc_cost in FP64 on those values, v is FP32.  ore is a step in g: it has
 * no gradient.
 *
 * mm_relaxed_forward: x_dev[B][T] FP32 -> *J_dev, npv_dev[S] and ore_t_dev[T][S]
 * (FP64, device).  ore_t_dev is the per-period checkpoint O[t][s] that the
 * adjoint reads.  The products run on the tensor cores as TF32 with every
 * FP32 operand split into hi + lo (FP32-accurate), accumulated in FP32 over
 * each CTA's range of blocks; the ranges' sums are added by compensated FP32
 * in a fixed order, the penalty, NPV_s and J in FP64 (deterministic).
 * mm_relaxed_backward: given the forward's npv_dev and ore_t_dev and the
 * upstream gradient *gJ_dev (FP64, device), writes gx_dev[B][T] = dJ/dx and,
 * if gg_dev is not NULL, gg_dev[B][S] = dJ/dg (FP32, device).  Where every
 * NPV_s is equal the std term contributes no gradient.  When npv_dev and
 * ore_t_dev are the buffers the model's last mm_relaxed_forward wrote, with
 * the same beta and m_ref, the adjoint reuses the coefficients that forward
 * left in model-owned memory (P_t'(O) and the scenario weights per unit gJ,
 * FP32) and launches no coefficient kernel; those buffers must then still hold
 * what that forward wrote.  Any other buffers: the coefficients are formed
 * from their contents first.
 * Both are asynchronous on the model's stream; the first call (or a larger
 * model) allocates model-owned scratch.  beta, m_ref > 0 (MM_ERR_INVALID_ARG
 * otherwise). */
mm_status mm_relaxed_forward(mm_model *m, const float *x_dev, const float *g_dev, double beta, double m_ref,
                             double *J_dev, double *npv_dev, double *ore_t_dev);
mm_status mm_relaxed_backward(mm_model *m, const float *x_dev, const float *g_dev, double beta, double m_ref,
                              const double *npv_dev, const double *ore_t_dev, const double *gJ_dev,
                              float *gx_dev, float *gg_dev);

/* The relaxed gradient as a first-order prior over candidate moves: at the
 * model's current schedule read as the one-hot x (x[b][t] = 1 at b's period,
 * none when unmined), moving block b from t1 to t2 changes x by -1 at (b, t1)
 * and +1 at (b, t2), so for the gradient gx_dev[B][T] = dJ/dx at that x
 *   shift b1: t1 -> t2 : prior = gx[b1][t2] - gx[b1][t1],
 *   swap b1 (t1) with b2 (t2): prior = (gx[b1][t2] - gx[b1][t1])
 *                                    + (gx[b2][t1] - gx[b2][t2]),
 * with gx[b][T] read as 0 (unmined).  prior_dev[n] (FP32, device); a bad move
 * gets -infinity and raises the sticky MM_ERR_BAD_MOVE.  A ranking aid only:
 * feasibility and the exact delta stay with mm_eval_moves.  Asynchronous. */
mm_status mm_relaxed_move_prior(mm_model *m, const float *gx_dev, const mm_move *moves_dev, int64_t n,
                                float *prior_dev);

/* ---- Precision study: FP32 shadow accumulators (no counterpart in the paper) ----
 * The model keeps its running per-period, per-scenario metal and NPV
 * contributions and NPV_s in FP64 because their drift accumulates over many
 * accepted moves.  mm_set_fp32_shadow(m, 1) adds the same running totals kept
 * in FP32 beside them (initialised from the current FP64 state, re-initialised
 * by every mm_schedule_set, updated by every apply with the same formulas in
 * FP32), so that the drift of the two can be compared against a full FP64
 * recomputation; 0 frees them.  Allocates; synchronising when freeing.
 * mm_get_fp32_shadow_npv writes the FP32 NPV_s as doubles to npv_host[S]
 * (synchronising; MM_ERR_STATE when the shadow is off). */
mm_status mm_set_fp32_shadow(mm_model *m, int32_t enable);
mm_status mm_get_fp32_shadow_npv(mm_model *m, double *npv_host);

/* Message of the last failing call on this thread ("" if none). */
const char *mm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MM_H */
