// Internal definitions of the move-evaluation engine (device state, launch
// helpers).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "mm.h"

namespace mm {

constexpr int kMaxS = 1024;       // scenarios per model
constexpr int kMaxT = 254;        // periods; the period byte value T means unmined
constexpr int kCtabMaxT = 64;     // the period-pair table is kept for T <= this
constexpr int kTopkMax = 1024;    // largest k of mm_topk
constexpr int kHistBits = 12;     // top-k coarse histogram over the key's top bits
constexpr int kHistBins = 1 << kHistBits;

// Sticky device status bits, read and cleared by synchronising calls.
enum : uint32_t { kStBadMove = 1u, kStTimeout = 2u };

// Outcome of an apply, written by the device.
struct ApplyResult {
    int32_t applied;   // 1 if the move was applied
    int32_t status;    // mm_status of the apply
    double mean, std;  // NPV mean / population std over scenarios after it
};

// Packed per-block schedule word read by the evaluator with one 4-byte load:
//   bits 0-7 period x_b, bits 8-15 lo_b = max period over direct predecessors
//   (0 if none), bits 16-23 hi_b = min period over direct successors (T if none).
// A shift of b to t' satisfies every arc at b iff lo_b <= t' <= hi_b.
__host__ __device__ inline uint32_t blk_pack(uint32_t t, uint32_t lo, uint32_t hi) {
    return t | (lo << 8) | (hi << 16);
}
__host__ __device__ inline uint32_t blk_period(uint32_t w) { return w & 0xffu; }
__host__ __device__ inline uint32_t blk_lo(uint32_t w) { return (w >> 8) & 0xffu; }
__host__ __device__ inline uint32_t blk_hi(uint32_t w) { return (w >> 16) & 0xffu; }

// Top-k scratch owned by a model (or by the caller-free static variant).
struct TopkScratch {
    uint32_t *hist = nullptr;      // [kHistBins] coarse histogram, zero between calls
    uint64_t *sure = nullptr;      // [kTopkMax] keys above the cut-off bin
    uint64_t *maybe = nullptr;     // [cap_maybe] keys inside the cut-off bin
    uint32_t *ctl = nullptr;       // [8] tickets, counters, cut-off
    int64_t cap_maybe = 0;
};

}  // namespace mm

struct mm_model {
    int32_t B = 0, S = 0, T = 0, S_pad = 0, W = 0;
    int32_t R = 0;        // row stride (floats) of the combined value/ore rows
    int32_t ore_off = 0;  // float index of the first ore word in a row (4 * ceil(S/4))
    int32_t nx = 0, ny = 0, nz = 0;   // grid of the 1-5 pattern, or 0 (CSR)
    int32_t uniform_mass = 0;
    uint32_t m_uniform = 0;
    double price = 0, recovery = 0, mining_cost = 0, proc_cost = 0;
    double shortfall_pen = 0, excess_pen = 0, discount_rate = 0, lambda = 0;
    cudaStream_t stream = nullptr;
    int has_schedule = 0;
    int num_sms = 148;
    size_t l2_bytes = 126u << 20;  // L2 size (cudaDevAttrL2CacheSize)
    int max_smem_optin = 227 * 1024;  // per-CTA shared-memory limit (opt-in)
    int team = 0;          // evaluator tile: lanes per move (0 = default)
    int ctas_per_sm = 0;   // evaluator grid: CTAs per SM (0 = occupancy maximum)
    int stages = -1;       // evaluator row staging: -1 default, 0 direct loads, 1..4 bulk-copy pipeline depth
    int prefetch = -1;     // direct loads: batches prefetched into L1 ahead (-1 default)
    std::map<const void *, size_t> smem_attr;  // dynamic shared-memory limit raised per kernel

    std::vector<double> h_disc;      // [T+1] d_t in FP64, d_T = 0
    std::vector<uint64_t> h_cap;     // [T]
    std::vector<uint64_t> h_target;  // [T]

    // device state
    uint32_t *mass = nullptr;    // [B]
    double *grade = nullptr;     // [B][S]
    float *val = nullptr;        // [B+1][R] rows: S FP32 values, 0 up to ore_off, W ore words, 0 (row B all 0);
                                 // with weights sigma the values are the ore processing margins (0 for waste)
    uint32_t *blk = nullptr;     // [B] packed period / lo / hi
    int32_t *pred_ptr = nullptr, *pred_idx = nullptr;  // CSR (device) when nx == 0
    int32_t *succ_ptr = nullptr, *succ_idx = nullptr;
    int32_t *order = nullptr;    // [B] blocks sorted by period (schedule_set)
    int32_t *porder = nullptr;   // [T+2] offsets of each period in order
    int4 *accum_chunk = nullptr;     // schedule_set: chunks of one period's blocks, (period, begin, end, 0) in order
    int32_t *accum_cbase = nullptr;  // [T+1] first chunk of each period
    int64_t *accum_ore = nullptr;    // [chunks][S] chunk partial ore tonnage
    double *accum_met = nullptr;     // [chunks][S] chunk partial metal
    int64_t *accum_mass = nullptr;   // [chunks] chunk mined tonnage
    int32_t accum_chunk_len = 0, accum_max_chunks = 0;
    int64_t *minedT = nullptr;   // [T+1]
    int64_t *oreT = nullptr;     // [T+1][S]  (row T stays 0)
    double *metal = nullptr;     // [T][S]    grams in situ of ore
    double *npv = nullptr;       // [S]
    double *contrib = nullptr;   // [T][S]    d_t (cash - penalty) per period
    float *tab = nullptr;        // [2][T+1][S_pad]  Pout, Pin
    float *tabc = nullptr;       // [T+1][4] Pout / Pin of a period when the deviation is far from the target
    float *ctab = nullptr;       // [T+1][T+1][S_pad] Pout[a] + Pin[b] (FP32 sum); T <= kCtabMaxT only
    float *ddt = nullptr;        // [(T+1)*(T+1)]    d_{t'} - d_t  (index t*(T+1)+t')
    double *disc = nullptr;      // [T+1]
    double *sig = nullptr;       // [T][S] uncertainty weights sigma(s,t) of Eq. 12 (nullptr: none)
    float *dwt = nullptr;        // [T+1][T+1][S_pad] sigma(s,b) d_b - sigma(s,a) d_a (FP64, rounded once), with weights
    uint64_t *cap = nullptr;     // [T+1]  cap[T] = max
    uint64_t *target = nullptr;  // [T+1]
    uint32_t *status = nullptr;  // sticky bits
    mm::ApplyResult *apply_res = nullptr;       // device
    mm::ApplyResult *apply_res_host = nullptr;  // pinned host mirror
    uint32_t *status_host = nullptr;            // pinned
    mm::TopkScratch topk;
    uint64_t *step_cta = nullptr;    // fused search step: [step_max_ctas][32] published keys
    uint64_t *step_grp = nullptr;    // [step_max_ctas][32] merged lists of groups of CTAs
    int4 *step_cinf = nullptr;       // [step_max_ctas] move record of each CTA list's best key
    int4 *step_ginf = nullptr;       // [step_max_ctas] move record of each group list's best key
    uint32_t *step_tick = nullptr;   // [step_max_ctas + 1] group tickets, then the final ticket (zero between launches)
    int4 *pending = nullptr;         // the move whose FP64 update a fused step left due: (b1, b2 or B,
                                     // t1 | t2 << 8, due); done by the next step's CTAs (a share of the
                                     // scenarios each) or by settle_money
    int money_due = 0;               // host: a fused step with apply was issued since the last settle
    int test_stall = 0;              // test-only (MM_TEST_STALL_BULK_WAIT at create): every bulk-copy stage
                                     // expects 16 bytes it never receives and waits about 1 ms, so the
                                     // evaluator's timeout path runs without any fault
    int test_stall_relax = 0;        // test-only (MM_TEST_STALL_RELAXED at create), one-shot: the next relaxed
                                     // forward's stage barriers expect one arrival nobody makes and every wait
                                     // of that launch gives up after about 1 ms, so its timeout path runs
                                     // without any fault
    int step_max_ctas = 0;
    void *step_event = nullptr;      // cudaEvent_t recorded between the step's two launches (timing hook)
    float *shadow32 = nullptr;       // FP32 shadow accumulators: metal [T][S], contrib [T][S], npv [S]
    float *relax_scratch = nullptr;  // relaxed objective: range partials and terms / adjoint coefficients
    uint32_t *relax_tick = nullptr;  // relaxed forward: ticket of its finishing launch (zero between launches)
    size_t relax_scratch_floats = 0;
    // relaxed forward -> adjoint: P_t'(O[t][s]) [T][S] and the scenario weights
    // w_s / gJ [S] (FP32) the last forward prepared, for the outputs and
    // smoothing it was called with
    float *relax_coef = nullptr;
    size_t relax_coef_floats = 0;
    const double *rc_npv = nullptr, *rc_ore = nullptr;
    double rc_beta = 0.0, rc_mref = 0.0;
};

namespace mm {

// Thread-local error message and status helpers.
mm_status set_error(mm_status st, const char *fmt, ...);
mm_status cuda_status(cudaError_t e, const char *what);
mm_status check_launch(const char *what);
mm_status read_sticky(mm_model *m);  // synchronises, clears and maps the sticky bits
mm_status sticky_status(mm_model *m, uint32_t st);  // maps and clears sticky bits already read back

// Kernels and launchers shared between translation units.
mm_status rebuild_tables(mm_model *m);                     // Pout/Pin from oreT
// Launch the FP64 update a fused step left due (metal, net cash, NPV_s), if
// any; every host path that reads or changes those totals calls it first.
mm_status settle_money(mm_model *m, cudaStream_t stream = nullptr);  // nullptr: the model's stream
// Outputs of the fused search step (top-k of the batch, optional apply).
struct StepOut {
    int32_t k, apply;
    int32_t *idx;
    float *top;
    int32_t *count;
    int grid;  // set by eval_launch: CTAs that publish a list
};
mm_status eval_launch(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas, float *mean,
                      float *delta, int32_t options, int team, int ctas_per_sm, int stages, const StepOut *step,
                      const uint32_t *pmoves = nullptr);  // pmoves: the batch in the compact 4-byte form
int default_team(int S);
bool sigma_fast_ok(const mm_model *m, int options);  // the weighted fast form (and fused step) applies
// Top-k for k <= 32 through per-CTA warp lists and the step finisher.
mm_status topk_small_launch(mm_model *m, const float *score, const uint8_t *feas, int64_t n, int32_t k, int32_t *idx,
                            float *top, int32_t *count);
mm_status topk_launch(const float *score, const uint8_t *feas, int64_t n, int32_t k, int32_t *idx,
                      float *top, int32_t *count, TopkScratch &scr, int num_sms, cudaStream_t st);
mm_status topk_scratch_reserve(TopkScratch &scr, int64_t n);
void topk_scratch_free(TopkScratch &scr);

}  // namespace mm

#define MM_CUDA_TRY(expr, what)                              \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return mm::cuda_status(e_, what); \
    } while (0)
