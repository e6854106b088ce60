// Batched move evaluation (the hot path): per (move, scenario) NPV delta,
// exact feasibility flag, scenario reduction to mean - lambda*std.
//
// Work mapping (k_eval_tiled, mm_eval_tiled.cuh): a CTA decodes a tile of 256
// moves with one thread per move, then "teams" of TEAM lanes (4, 8, 16 or 32)
// evaluate one move each; lane l of a team owns scenario quads q = l,
// l + TEAM, ... (four scenarios per quad, one 16-byte load per row), so a
// team reads each moved block's value row with coalesced 128-bit loads.  The
// scenario mean and variance are reduced with xor-shuffles inside the team,
// two-pass (the deviations stay in registers), so a structural zero
// (identical blocks, a no-op) is exactly 0.
//
// Per-(move, scenario) arithmetic with uniform block mass m (all workloads):
//   block b1 moves t1 -> t2 (and, for a swap, b2 moves t2 -> t1)
//   delta_s = (v1_s - v2_s) * (d_t2 - d_t1)
//           + [o1 & !o2] (Pout[t1][s] + Pin[t2][s])
//           + [o2 & !o1] (Pin[t1][s] + Pout[t2][s])
// where v2 = 0, o2 = 0 for a shift (its partner is the all-zero row B), and Pout/Pin are the NPV changes of
// removing/adding one block of ore tonnage in (t, s), built in FP64 from the
// exact integer ore tonnage (so no penalty is formed as a difference of large
// FP32 numbers).  With unequal masses a general kernel forms the penalty
// change per (move, scenario) from the integer tonnages instead.
#include <map>
#include <mutex>
#include <utility>

#include "mm_eval_tiled.cuh"

namespace mm {

using EvalFn = void (*)(EvalArgs);
EvalFn pick_tiled_plain(int team, int qmax, bool delta, bool tsm, bool tma);
EvalFn pick_tiled_kahan(int team, int qmax, bool delta, bool tsm, bool tma);
EvalFn pick_fast_plain(int team, int kf, bool tail, bool delta);
EvalFn pick_fast_kahan(int team, int kf, bool tail, bool delta);
EvalFn pick_fast_sigma(int team, int kf, bool tail, bool delta);
EvalFn pick_step_sigma(int team, int kf, bool tail);

// The weighted fast form applies: equal masses, the period-pair table kept,
// S % 4 == 0 and 1..4 full quad iterations per lane at the model's team.
bool sigma_fast_ok(const mm_model *m, int options) {
    if (!m->sig || !m->uniform_mass || !m->ctab || m->S % 4 != 0) return false;
    if (options & (MM_EVAL_KAHAN | MM_EVAL_GENERIC)) return false;
    const int team = m->team > 0 ? m->team : default_team(m->S);
    const int kf = ((m->S + 3) / 4) / team;
    return kf >= 1 && kf <= 4;
}
EvalFn pick_step(int team, bool fast, int kf, bool tail, int qmax, bool tsm);
ApplyArgs apply_args(mm_model *m);

// General evaluator (unequal block masses, and every weighted model the fast
// form does not take): one warp per move, one lane per scenario, penalty
// change from the exact integer ore tonnages:
//   dO = m2*o2 - m1*o1 enters period t1 and leaves period t2;
//   delta_s = (v1 - v2)(d_t2 - d_t1) + d_t1 (pen(x1) - pen(x1 + dO)) + d_t2 (pen(x2) - pen(x2 - dO)).
// With uncertainty weights (Eq. 12) v is the ore margin, d_t2 - d_t1 becomes
// the scenario's weighted difference dwt[t1][t2][s], and the mining cost adds
// -mc (m1 - m2)(d_t2 - d_t1), formed in FP64 per move.
__device__ __forceinline__ double pen_diff_g(int64_t x0, int64_t x1, double a, double e) {
    int64_t s0 = x0 < 0 ? -x0 : 0, s1 = x1 < 0 ? -x1 : 0;
    int64_t e0 = x0 > 0 ? x0 : 0, e1 = x1 > 0 ? x1 : 0;
    return a * (double)(s0 - s1) + e * (double)(e0 - e1);
}

template <bool DELTA>
__global__ void __launch_bounds__(256) k_eval_general(EvalArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int S = A.S, T1 = A.T + 1;
    for (int64_t i = warp_gid; i < A.n; i += nwarps) {
        const int2 mv = __ldg(A.moves + i);
        const MoveView v = decode_move(
            mv, A.tp, [&](int32_t b) { return __ldg(A.blk + b); }, [&](int32_t b) { return __ldg(A.mass + b); },
            [&](uint32_t t) { return A.minedT[t]; }, [&](uint32_t t) { return A.cap[t]; });
        const bool work = v.valid && !v.noop;
        float sum = 0.0f;
        float dl[kMaxS / 32];
        const float dd = work ? __ldg(A.ddt + v.t1 * T1 + v.t2) : 0.0f;
        const bool sig = A.dwt != nullptr;
        const float *dwrow = sig ? A.dwt + ((size_t)v.t1 * T1 + v.t2) * A.S_pad : nullptr;
        float cmv = 0.0f;
        if (sig && work)
            cmv = (float)(-A.mc * ((double)v.m1 - (v.swap ? (double)v.m2 : 0.0)) * (A.disc[v.t2] - A.disc[v.t1]));
#pragma unroll 4
        for (int k = 0; k < kMaxS / 32; k++) {
            const int s = lane + 32 * k;
            float x = 0.0f;
            if (work && s < S) {
                const float *row1 = A.val + (int64_t)v.b1 * A.R;
                const uint32_t o1 = (__ldg(reinterpret_cast<const uint32_t *>(row1 + A.ore_off) + (s >> 5)) >> (s & 31)) & 1u;
                const float v1 = __ldg(row1 + s);
                uint32_t o2 = 0;
                float v2 = 0.0f;
                if (v.swap) {
                    const float *row2 = A.val + (int64_t)v.b2 * A.R;
                    o2 = (__ldg(reinterpret_cast<const uint32_t *>(row2 + A.ore_off) + (s >> 5)) >> (s & 31)) & 1u;
                    v2 = __ldg(row2 + s);
                }
                const int64_t dO = (int64_t)(o2 ? v.m2 : 0) - (int64_t)(o1 ? v.m1 : 0);
                double p = 0.0;
                if (dO != 0) {
                    if (v.t1 < (uint32_t)A.T) {
                        int64_t x1 = A.oreT[(int64_t)v.t1 * S + s] - (int64_t)A.target[v.t1];
                        p += A.disc[v.t1] * pen_diff_g(x1, x1 + dO, A.a, A.e);
                    }
                    if (v.t2 < (uint32_t)A.T) {
                        int64_t x2 = A.oreT[(int64_t)v.t2 * S + s] - (int64_t)A.target[v.t2];
                        p += A.disc[v.t2] * pen_diff_g(x2, x2 - dO, A.a, A.e);
                    }
                }
                x = sig ? fmaf(v1 - v2, __ldg(dwrow + s), (float)p + cmv) : fmaf(v1 - v2, dd, (float)p);
            }
            dl[k] = x;
            sum += x;
            if (32 * (k + 1) >= S) break;
        }
        const float invS = 1.0f / (float)S;
        const float mu = team_sum<32>(sum) * invS;
        float var = 0.0f;
#pragma unroll 4
        for (int k = 0; k < kMaxS / 32; k++) {
            const int s = lane + 32 * k;
            if (s < S) {
                const float dv = dl[k] - mu;
                var = fmaf(dv, dv, var);
            }
            if (32 * (k + 1) >= S) break;
        }
        var = team_sum<32>(var);
        const float sd = sqrtf(var * invS);
        if (lane == 0) {
            float sc = !v.valid ? -INFINITY : (work ? mu - A.lambda * sd : 0.0f);
            if (!v.valid) atomicOr(A.status, kStBadMove);
            A.score[i] = sc;
            A.feas[i] = v.feasible ? 1 : 0;
            if (A.mean) A.mean[i] = work ? mu : 0.0f;
        }
        if (DELTA) {
            for (int k = 0; k < kMaxS / 32; k++) {
                const int s = lane + 32 * k;
                if (s < S) A.delta[i * (int64_t)S + s] = dl[k];
                if (32 * (k + 1) >= S) break;
            }
        }
    }
}

// ------------------------------------------------------------ dispatch

// Team size: the smallest power of two in 4..32 that keeps quads per lane
// <= 4, else 32 lanes with up to 8 quads per lane.
int default_team(int S) {
    int nq = (S + 3) / 4;
    for (int team = 4; team <= 32; team *= 2)
        if ((nq + team - 1) / team <= 4) return team;
    return 32;
}

// Evaluator arguments for a batch of n moves on model m (the step fields
// cleared).
StepLists step_lists(mm_model *m, int grid) {
    StepLists L;
    L.cta = m->step_cta;
    L.grp = m->step_grp;
    L.cinf = m->step_cinf;
    L.ginf = m->step_ginf;
    L.tick = m->step_tick;
    L.final_slot = m->step_max_ctas;
    int g = 1;
    while (g * g < grid) g++;  // about sqrt(grid) CTAs per group and groups
    L.grp_size = g;
    return L;
}

EvalArgs eval_args(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas, float *mean,
                   float *delta) {
    EvalArgs A;
    A.moves = reinterpret_cast<const int2 *>(moves);
    A.pmoves = nullptr;
    A.n = n;
    A.score = score; A.feas = feas; A.mean = mean; A.delta = delta;
    A.val = m->val; A.blk = m->blk; A.mass = m->mass;
    A.tab = m->tab; A.ctab = m->ctab; A.ddt = m->ddt; A.minedT = m->minedT; A.cap = m->cap;
    A.oreT = m->oreT; A.target = m->target; A.disc = m->disc; A.dwt = m->dwt;
    A.status = m->status;
    A.tp.B = m->B; A.tp.T = m->T; A.tp.nx = m->nx; A.tp.ny = m->ny; A.tp.nz = m->nz;
    A.tp.pred_ptr = m->pred_ptr; A.tp.pred_idx = m->pred_idx; A.tp.succ_ptr = m->succ_ptr; A.tp.succ_idx = m->succ_idx;
    A.S = m->S; A.S_pad = m->S_pad; A.W = m->W; A.T = m->T; A.R = m->R; A.ore_off = m->ore_off;
    A.m_uniform = m->m_uniform;
    A.nstage = 0;
    A.tx_extra = m->test_stall ? 16u : 0u;
    A.wait_cycles = m->test_stall ? kTestWaitCycles : kWaitCycles;
    A.dd_smem = (size_t)(m->T + 1) * (m->T + 1) * sizeof(float) <= kDdSmemMax ? 1 : 0;
    A.prefetch = m->prefetch >= 0 ? m->prefetch : ((size_t)m->B * m->R * sizeof(float) > m->l2_bytes ? kPrefetchDram : 0);

    A.lambda = (float)m->lambda;
    A.a = m->shortfall_pen; A.e = m->excess_pen; A.mc = m->mining_cost;
    A.mcm = (float)(m->mining_cost * (double)m->m_uniform);
    A.qpl = 0;
    A.tail = StepTail{};
    A.tail.L = step_lists(m, 1);
    A.tail.n = n;
    A.tail.status = m->status;
    A.tail.moves = A.moves;
    return A;
}

// Resident CTAs per SM of an evaluator, cached so that calls captured into a
// CUDA graph make no occupancy query.
static mm_status eval_occupancy(EvalFn fn, int threads, size_t smem, int *per_sm) {
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair((const void *)fn, smem);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *per_sm = it->second;
        return MM_OK;
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads, smem);
    if (e != cudaSuccess) return cuda_status(e, "occupancy query");
    if (*per_sm < 1) *per_sm = 1;
    cache[key] = *per_sm;
    return MM_OK;
}

mm_status eval_launch(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas, float *mean,
                      float *delta, int32_t options, int team, int ctas_per_sm, int stages, const StepOut *step,
                      const uint32_t *pmoves) {
    EvalArgs A = eval_args(m, moves, n, score, feas, mean, delta);
    A.pmoves = pmoves;
    // the fused step runs one CTA of kStepThreads per SM (its top-k lists meet
    // in one level); evaluation-only launches several CTAs of kEvalThreads
    const int nt = step ? kStepThreads : kEvalThreads;
    if (step) {
        A.tail.k = step->k;
        A.tail.idx_out = step->idx;
        A.tail.top_out = step->top;
        A.tail.count_out = step->count;
        A.tail.do_apply = step->apply;
        A.tail.ap = apply_args(m);  // the first CTA to finish also settles the previous step's FP64 update
        A.tail.pending = m->pending;
        stages = 0;  // the fused step runs on direct loads
    }
    const bool kahan = (options & MM_EVAL_KAHAN) != 0;
    const bool want_delta = delta != nullptr;
    if (m->sig && step && !sigma_fast_ok(m, options))
        return set_error(MM_ERR_INVALID_ARG, "the fused step takes uncertainty weights in the fast form only");
    if (sigma_fast_ok(m, options) && (team <= 0 || team == (m->team > 0 ? m->team : default_team(m->S)))) {
        // weighted fast form (direct loads), evaluation or the fused step
        if (team <= 0) team = default_team(m->S);
        const int nq = (m->S + 3) / 4, kf = nq / team;
        EvalFn fn = step ? pick_step_sigma(team, kf, nq % team != 0) : pick_fast_sigma(team, kf, nq % team != 0, want_delta);
        if (fn) {
            const int T1 = m->T + 1;
            const size_t smem = (((A.dd_smem ? (size_t)T1 * T1 * sizeof(float) : 0) + 15) & ~(size_t)15) +
                                2 * (size_t)T1 * sizeof(int64_t);
            if (m->smem_attr[(const void *)fn] < smem) {
                cudaFuncAttributes fa;
                cudaError_t e = cudaFuncGetAttributes(&fa, fn);
                if (e != cudaSuccess) return cuda_status(e, "evaluator attributes");
                if (fa.sharedSizeBytes + smem > 48 * 1024) {
                    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (e != cudaSuccess) return cuda_status(e, "set evaluator shared memory");
                }
                m->smem_attr[(const void *)fn] = smem;
            }
            int per_sm = step ? 0 : ctas_per_sm;
            if (per_sm <= 0) {
                const mm_status os = eval_occupancy(fn, nt, smem, &per_sm);
                if (os != MM_OK) return os;
            }
            A.qpl = (nq + team - 1) / team;
            const int64_t chunks = (n + kChunk - 1) / kChunk;
            int64_t blocks = (chunks + nt / 32 - 1) / (nt / 32);
            int64_t grid_cap = (int64_t)m->num_sms * per_sm;
            if (step && grid_cap > m->step_max_ctas) grid_cap = m->step_max_ctas;
            if (blocks > grid_cap) blocks = grid_cap;
            if (blocks < 1) blocks = 1;
            if (step) const_cast<StepOut *>(step)->grid = (int)blocks;
            A.tail.L = step_lists(m, (int)blocks);
            fn<<<(unsigned)blocks, nt, smem, m->stream>>>(A);
            return check_launch("k_eval_tiled");
        }
    }
    if (m->sig && step) return set_error(MM_ERR_INVALID_ARG, "no weighted step kernel for this tile");
    if (!m->uniform_mass || m->sig) {
        if (pmoves) return set_error(MM_ERR_INVALID_ARG, "compact moves need the tiled evaluator");
        EvalFn fn = want_delta ? k_eval_general<true> : k_eval_general<false>;
        int64_t blocks = (n + 7) / 8;
        int64_t cap_blocks = (int64_t)m->num_sms * 8;
        if (blocks > cap_blocks) blocks = cap_blocks;
        if (blocks < 1) blocks = 1;
        fn<<<(unsigned)blocks, 256, 0, m->stream>>>(A);
        return check_launch("k_eval_general");
    }
    if (team <= 0) team = default_team(m->S);
    const int nq = (m->S + 3) / 4;
    const int qpl = (nq + team - 1) / team;
    int qmax = 1;
    while (qmax < qpl) qmax <<= 1;
    A.qpl = qpl;
    const int T1 = m->T + 1;
    const size_t tab_bytes = (size_t)2 * T1 * m->S_pad * sizeof(float);
    const size_t small = (((A.dd_smem ? (size_t)T1 * T1 * sizeof(float) : 0) + 15) & ~(size_t)15) +
                         2 * (size_t)T1 * sizeof(int64_t);
    if (stages < 0) stages = kDefaultStages;
    if (stages > kMaxStages) stages = kMaxStages;
    const bool tma = stages > 0;
    // fast form: S % 4 == 0, floor(NQ / team) full quad iterations known at
    // compile time, period-pair table read from global memory
    const int kf = nq / team;
    const bool tail = nq % team != 0;
    const bool fast_ok = !tma && m->ctab && m->S % 4 == 0 && !(options & MM_EVAL_GENERIC) && kf >= 1 && kf <= 4;
    // otherwise the Pout / Pin tables are staged in shared memory when small
    const bool tsm = !fast_ok && tab_bytes <= 64 * 1024;
    A.nstage = stages;
    size_t smem = (tsm ? tab_bytes : 0) + small;
    if (tma) {
        // the static shared arrays of the kernel take ~12 KB; keep a margin
        const size_t base = ((smem + 127) & ~(size_t)127);
        const size_t per_stage = (size_t)(kEvalThreads / 32) * (32 / team) * 2 * m->R * sizeof(float);
        while (stages > 1 && base + stages * per_stage + 16 * 1024 > (size_t)m->max_smem_optin) stages--;
        if (base + stages * per_stage + 16 * 1024 > (size_t)m->max_smem_optin) stages = 0;
        if (stages > 0) smem = base + stages * per_stage;
    }
    const bool use_tma = stages > 0;
    A.nstage = stages;
    EvalFn fn = nullptr;
    if (step) {
        fn = pick_step(team, fast_ok, kf, tail, qmax, tsm);
    } else {
        if (fast_ok)
            fn = kahan ? pick_fast_kahan(team, kf, tail, want_delta) : pick_fast_plain(team, kf, tail, want_delta);
        if (!fn)
            fn = kahan ? pick_tiled_kahan(team, qmax, want_delta, tsm, use_tma)
                       : pick_tiled_plain(team, qmax, want_delta, tsm, use_tma);
    }
    if (!fn) return set_error(MM_ERR_INVALID_ARG, "no evaluator for team %d with %d quads per lane", team, qpl);
    // the 48 KB default covers static + dynamic shared memory; a kernel whose
    // static part (up to ~32 KB with the in-launch apply) and dynamic part
    // exceed it opts in (once per kernel and size)
    if (m->smem_attr[(const void *)fn] < smem) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, fn);
        if (e != cudaSuccess) return cuda_status(e, "evaluator attributes");
        if (fa.sharedSizeBytes + smem > 48 * 1024) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_status(e, "set evaluator shared memory");
        }
        m->smem_attr[(const void *)fn] = smem;
    }
    int per_sm = step ? 0 : ctas_per_sm;
    if (per_sm <= 0) {
        const mm_status os = eval_occupancy(fn, nt, smem, &per_sm);
        if (os != MM_OK) return os;
    }
    const int64_t chunks = (n + kChunk - 1) / kChunk;
    int64_t blocks = (chunks + nt / 32 - 1) / (nt / 32);
    int64_t grid_cap = (int64_t)m->num_sms * per_sm;
    if (step && grid_cap > m->step_max_ctas) grid_cap = m->step_max_ctas;
    if (blocks > grid_cap) blocks = grid_cap;
    if (blocks < 1) blocks = 1;
    if (step) const_cast<StepOut *>(step)->grid = (int)blocks;
    A.tail.L = step_lists(m, (int)blocks);
    fn<<<(unsigned)blocks, nt, smem, m->stream>>>(A);
    return check_launch("k_eval_tiled");
}

}  // namespace mm

using namespace mm;

static mm_status eval_check(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    if (n < 0) return set_error(MM_ERR_INVALID_ARG, "negative move count");
    if (n > 0 && (!moves || !score || !feas)) return set_error(MM_ERR_INVALID_ARG, "NULL output or move pointer");
    if (((uintptr_t)moves & 7u) != 0) return set_error(MM_ERR_INVALID_ARG, "moves must be 8-byte aligned");
    return MM_OK;
}

extern "C" {

mm_status mm_eval_moves(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas, float *mean) {
    mm_status st = eval_check(m, moves, n, score, feas);
    if (st != MM_OK || n == 0) return st;
    return eval_launch(m, moves, n, score, feas, mean, nullptr, MM_EVAL_PLAIN, m->team, m->ctas_per_sm, m->stages,
                       nullptr);
}

mm_status mm_set_tile(mm_model *m, int32_t team, int32_t ctas_per_sm, int32_t stages, int32_t prefetch) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (team != 0 && team != 4 && team != 8 && team != 16 && team != 32)
        return set_error(MM_ERR_INVALID_ARG, "team must be 0, 4, 8, 16 or 32");
    if (team != 0 && ((m->S + 3) / 4 + team - 1) / team > 8)
        return set_error(MM_ERR_INVALID_ARG, "team %d leaves more than 8 quads per lane at S = %d", team, m->S);
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return set_error(MM_ERR_INVALID_ARG, "ctas_per_sm out of range");
    if (stages < -1 || stages > kMaxStages) return set_error(MM_ERR_INVALID_ARG, "stages must be -1..%d", kMaxStages);
    m->team = team;
    m->ctas_per_sm = ctas_per_sm;
    if (prefetch < -1 || prefetch > 8) return set_error(MM_ERR_INVALID_ARG, "prefetch must be -1..8");
    m->stages = stages;
    m->prefetch = prefetch;
    return MM_OK;
}

mm_status mm_eval_moves_ex(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas, float *mean,
                           float *delta, int32_t options) {
    mm_status st = eval_check(m, moves, n, score, feas);
    if (st != MM_OK || n == 0) return st;
    if (options & ~(MM_EVAL_KAHAN | MM_EVAL_GENERIC))
        return set_error(MM_ERR_INVALID_ARG, "unknown option bits 0x%x", options);
    return eval_launch(m, moves, n, score, feas, mean, delta, options, m->team, m->ctas_per_sm, m->stages, nullptr);
}

}  // extern "C"

