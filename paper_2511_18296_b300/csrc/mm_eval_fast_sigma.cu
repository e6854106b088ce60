// Instantiations of the tiled evaluator's fast form with uncertainty weights
// (Eq. 12: the value term takes the per-scenario weighted discount difference
// of the move's period pair), plain FP32 tree sums.
#include "mm_eval_tiled.cuh"

namespace mm {

using EvalFn = void (*)(EvalArgs);

template <int TEAM, int KF, bool TAIL>
static EvalFn fast3(bool delta) {
    return delta ? k_eval_tiled<TEAM, 1, false, true, false, KF, TAIL, false, true>
                 : k_eval_tiled<TEAM, 1, false, false, false, KF, TAIL, false, true>;
}

template <int TEAM>
static EvalFn fast2(int kf, bool tail, bool delta) {
    switch (kf) {
        case 1: return tail ? fast3<TEAM, 1, true>(delta) : fast3<TEAM, 1, false>(delta);
        case 2: return tail ? fast3<TEAM, 2, true>(delta) : fast3<TEAM, 2, false>(delta);
        case 3: return tail ? fast3<TEAM, 3, true>(delta) : fast3<TEAM, 3, false>(delta);
        case 4: return tail ? fast3<TEAM, 4, true>(delta) : fast3<TEAM, 4, false>(delta);
    }
    return nullptr;
}

// The fused search step's weighted form (top-k and in-launch apply), one
// CTA of kStepThreads per SM.
template <int TEAM>
static EvalFn step2(int kf, bool tail) {
    switch (kf) {
        case 1: return tail ? k_eval_tiled<TEAM, 1, false, false, false, 1, true, true, true, kStepThreads>
                            : k_eval_tiled<TEAM, 1, false, false, false, 1, false, true, true, kStepThreads>;
        case 2: return tail ? k_eval_tiled<TEAM, 1, false, false, false, 2, true, true, true, kStepThreads>
                            : k_eval_tiled<TEAM, 1, false, false, false, 2, false, true, true, kStepThreads>;
        case 3: return tail ? k_eval_tiled<TEAM, 1, false, false, false, 3, true, true, true, kStepThreads>
                            : k_eval_tiled<TEAM, 1, false, false, false, 3, false, true, true, kStepThreads>;
        case 4: return tail ? k_eval_tiled<TEAM, 1, false, false, false, 4, true, true, true, kStepThreads>
                            : k_eval_tiled<TEAM, 1, false, false, false, 4, false, true, true, kStepThreads>;
    }
    return nullptr;
}

EvalFn pick_step_sigma(int team, int kf, bool tail) {
    switch (team) {
        case 4: return step2<4>(kf, tail);
        case 8: return step2<8>(kf, tail);
        case 16: return step2<16>(kf, tail);
        case 32: return step2<32>(kf, tail);
    }
    return nullptr;
}

EvalFn pick_fast_sigma(int team, int kf, bool tail, bool delta) {
    switch (team) {
        case 4: return fast2<4>(kf, tail, delta);
        case 8: return fast2<8>(kf, tail, delta);
        case 16: return fast2<16>(kf, tail, delta);
        case 32: return fast2<32>(kf, tail, delta);
    }
    return nullptr;
}

}  // namespace mm
