// The fused search step: instantiations of the evaluator's top-k variant
// (plain FP32 sums, no per-scenario output, one CTA of kStepThreads per SM;
// the batch's top k is selected and the best move applied by the CTA that
// finishes last, see step_finish), the list-based top-k for k <= 32, and the
// entry point.
#include "mm_eval_tiled.cuh"

namespace mm {

using EvalFn = void (*)(EvalArgs);

template <int TEAM, int KF, bool TAIL>
static EvalFn step_fast3() {
    return k_eval_tiled<TEAM, 1, false, false, false, KF, TAIL, true, false, kStepThreads>;
}

template <int TEAM>
static EvalFn step_fast2(int kf, bool tail) {
    switch (kf) {
        case 1: return tail ? step_fast3<TEAM, 1, true>() : step_fast3<TEAM, 1, false>();
        case 2: return tail ? step_fast3<TEAM, 2, true>() : step_fast3<TEAM, 2, false>();
        case 3: return tail ? step_fast3<TEAM, 3, true>() : step_fast3<TEAM, 3, false>();
        case 4: return tail ? step_fast3<TEAM, 4, true>() : step_fast3<TEAM, 4, false>();
    }
    return nullptr;
}

template <int TEAM, int QMAX>
static EvalFn step_gen2(bool tsm) {
    return tsm ? k_eval_tiled<TEAM, QMAX, false, false, true, 0, false, true, false, kStepThreads>
               : k_eval_tiled<TEAM, QMAX, false, false, false, 0, false, true, false, kStepThreads>;
}

template <int TEAM>
static EvalFn step_gen1(int qmax, bool tsm) {
    switch (qmax) {
        case 1: return step_gen2<TEAM, 1>(tsm);
        case 2: return step_gen2<TEAM, 2>(tsm);
        case 4: return step_gen2<TEAM, 4>(tsm);
        case 8: return step_gen2<TEAM, 8>(tsm);
    }
    return nullptr;
}

EvalFn pick_step(int team, bool fast, int kf, bool tail, int qmax, bool tsm) {
    if (fast) {
        switch (team) {
            case 4: return step_fast2<4>(kf, tail);
            case 8: return step_fast2<8>(kf, tail);
            case 16: return step_fast2<16>(kf, tail);
            case 32: return step_fast2<32>(kf, tail);
        }
        return nullptr;
    }
    switch (team) {
        case 4: return step_gen1<4>(qmax, tsm);
        case 8: return step_gen1<8>(qmax, tsm);
        case 16: return step_gen1<16>(qmax, tsm);
        case 32: return step_gen1<32>(qmax, tsm);
    }
    return nullptr;
}

// Standalone top-k for k <= 32: the same per-CTA lists as the fused step,
// built from stored scores and flags (four 32-key rounds in flight per warp).
__global__ void __launch_bounds__(kEvalThreads) k_topk_lists(const float *__restrict__ score,
                                                             const uint8_t *__restrict__ feas, int64_t n,
                                                             StepTail tail) {
    constexpr int NW = kEvalThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * NW, gw = (int64_t)blockIdx.x * NW + warp;
    const int64_t r0 = gw * n / nwarps, r1 = (gw + 1) * n / nwarps;
    uint64_t wtk = 0;
    for (int64_t c = r0; c < r1; c += 4 * 32) {
        float f[4];
        uint8_t ok[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = c + u * 32 + lane;
            ok[u] = i < r1 ? __ldg(feas + i) : 0;
            f[u] = i < r1 ? __ldg(score + i) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = c + u * 32 + lane;
            wtk = warp_topk_insert(wtk, (ok[u] && !isnan(f[u])) ? score_key(f[u], i) : 0ull);
        }
    }
    step_reduce(tail, wtk);
}

mm_status topk_small_launch(mm_model *m, const float *score, const uint8_t *feas, int64_t n, int32_t k, int32_t *idx,
                            float *top, int32_t *count) {
    int64_t blocks = (n + 2047) / 2048;
    if (blocks > (int64_t)m->num_sms * 2) blocks = (int64_t)m->num_sms * 2;
    if (blocks > m->step_max_ctas) blocks = m->step_max_ctas;
    if (blocks < 1) blocks = 1;
    StepTail tail{};
    tail.L = step_lists(m, (int)blocks);
    tail.k = k;
    tail.n = n;
    tail.status = m->status;
    tail.idx_out = idx;
    tail.top_out = top;
    tail.count_out = count;
    tail.do_apply = 0;
    tail.moves = nullptr;
    k_topk_lists<<<(unsigned)blocks, kEvalThreads, 0, m->stream>>>(score, feas, n, tail);
    return check_launch("k_topk_lists");
}

}  // namespace mm

using namespace mm;

static mm_status step_check(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    if (n < 0 || n > 0x7fffffffLL) return set_error(MM_ERR_INVALID_ARG, "move count out of range");
    if (n > 0 && (!moves || !score || !feas)) return set_error(MM_ERR_INVALID_ARG, "NULL output or move pointer");
    if (((uintptr_t)moves & 7u) != 0) return set_error(MM_ERR_INVALID_ARG, "moves must be 8-byte aligned");
    return MM_OK;
}

// The timing hook: the caller's event between a step's evaluation and apply
// (an external node while the stream is being captured).
static mm_status record_step_event(mm_model *m) {
    if (!m->step_event) return MM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MM_CUDA_TRY(cudaStreamIsCapturing(m->stream, &cs), "query stream capture");
    cudaEvent_t ev = static_cast<cudaEvent_t>(m->step_event);
    MM_CUDA_TRY(cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, m->stream, cudaEventRecordExternal)
                                                    : cudaEventRecord(ev, m->stream),
                "record the step event");
    return MM_OK;
}

// The step on a batch in either form (moves, or pmoves when packed; the
// compact form only where the whole step is one launch).
static mm_status search_step(mm_model *m, const mm_move *moves, const uint32_t *pmoves, bool packed, int64_t n,
                             int32_t k, int32_t apply, float *score, uint8_t *feas, int32_t *idx, float *top,
                             int32_t *count) {
    const char *name = packed ? "mm_search_step_packed" : "mm_search_step";
    if (k < 1 || k > 32) return set_error(MM_ERR_INVALID_ARG, "%s: k = %d outside 1..32", name, k);
    if (!idx || !top || !count) return set_error(MM_ERR_INVALID_ARG, "NULL top-k output");
    if (!m->uniform_mass)
        return set_error(MM_ERR_INVALID_ARG, "%s needs equal block masses (use the separate calls)", name);
    const bool weighted_split = m->sig && !sigma_fast_ok(m, MM_EVAL_PLAIN);
    // the final CTA of the evaluation launch applies the best move itself
    // when a CTA has a thread per scenario; otherwise a one-CTA launch follows
    const bool in_launch = apply && m->S <= kStepThreads;
    if (packed && (weighted_split || (apply && !in_launch)))
        return set_error(MM_ERR_INVALID_ARG,
                         "mm_search_step_packed: this model's step is not one launch (S = %d%s); use "
                         "mm_unpack_moves and mm_search_step",
                         m->S, weighted_split ? ", weights outside the fast form" : "");
    if (n == 0) {
        MM_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int32_t), m->stream), "clear count");
        return apply ? mm_apply_best(m, moves, 0, idx, count) : MM_OK;
    }
    mm_status st;
    if (weighted_split) {
        // uncertainty weights outside the weighted fast form: the separate
        // evaluation, top-k and apply launches
        st = eval_launch(m, moves, n, score, feas, nullptr, nullptr, MM_EVAL_PLAIN, m->team, m->ctas_per_sm, 0,
                         nullptr);
        if (st == MM_OK) st = mm_topk(m, score, feas, n, k, idx, top, count);
        if (st == MM_OK) st = record_step_event(m);
        return (st == MM_OK && apply) ? mm_apply_best(m, moves, n, idx, count) : st;
    }
    StepOut so{k, in_launch ? 1 : 0, idx, top, count, 0};
    st = eval_launch(m, moves, n, score, feas, nullptr, nullptr, MM_EVAL_PLAIN, m->team, m->ctas_per_sm, 0, &so,
                     pmoves);
    if (st != MM_OK) return st;
    // the launch's final CTA leaves the applied move's FP64 update due
    if (in_launch) m->money_due = 1;
    st = record_step_event(m);
    if (st != MM_OK) return st;
    return (apply && !in_launch) ? mm_apply_best(m, moves, n, idx, count) : MM_OK;
}

extern "C" mm_status mm_search_step(mm_model *m, const mm_move *moves, int64_t n, int32_t k, int32_t apply,
                                    float *score, uint8_t *feas, int32_t *idx, float *top, int32_t *count) {
    mm_status st = step_check(m, moves, n, score, feas);
    if (st != MM_OK) return st;
    return search_step(m, moves, nullptr, false, n, k, apply, score, feas, idx, top, count);
}

extern "C" mm_status mm_search_step_packed(mm_model *m, const uint32_t *packed, int64_t n, int32_t k, int32_t apply,
                                           float *score, uint8_t *feas, int32_t *idx, float *top, int32_t *count) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    if (n < 0 || n > 0x7fffffffLL) return set_error(MM_ERR_INVALID_ARG, "move count out of range");
    if ((int64_t)m->B + m->T + 1 > 65536)
        return set_error(MM_ERR_INVALID_ARG, "packed moves need B + T + 1 <= 65536 (B = %d, T = %d)", m->B, m->T);
    if (n > 0 && (!packed || !score || !feas)) return set_error(MM_ERR_INVALID_ARG, "NULL output or move pointer");
    if (((uintptr_t)packed & 3u) != 0) return set_error(MM_ERR_INVALID_ARG, "packed moves must be 4-byte aligned");
    return search_step(m, nullptr, packed, true, n, k, apply, score, feas, idx, top, count);
}

extern "C" mm_status mm_set_step_event(mm_model *m, void *cuda_event) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    m->step_event = cuda_event;
    return MM_OK;
}
