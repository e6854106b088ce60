// Instantiations of the tiled evaluator with plain FP32 tree sums
// (compiled as a separate translation unit so the builds run in parallel).
#include "mm_eval_tiled.cuh"

namespace mm {

using EvalFn = void (*)(EvalArgs);

template <int TEAM, int QMAX>
static EvalFn pick2(bool delta, bool tsm, bool tma) {
    if (tma) {
        if (delta) return tsm ? k_eval_tma<TEAM, QMAX, false, true, true> : k_eval_tma<TEAM, QMAX, false, true, false>;
        return tsm ? k_eval_tma<TEAM, QMAX, false, false, true> : k_eval_tma<TEAM, QMAX, false, false, false>;
    }
    if (delta) return tsm ? k_eval_tiled<TEAM, QMAX, false, true, true> : k_eval_tiled<TEAM, QMAX, false, true, false>;
    return tsm ? k_eval_tiled<TEAM, QMAX, false, false, true> : k_eval_tiled<TEAM, QMAX, false, false, false>;
}

template <int TEAM>
static EvalFn pick1(int qmax, bool delta, bool tsm, bool tma) {
    switch (qmax) {
        case 1: return pick2<TEAM, 1>(delta, tsm, tma);
        case 2: return pick2<TEAM, 2>(delta, tsm, tma);
        case 4: return pick2<TEAM, 4>(delta, tsm, tma);
        case 8: return pick2<TEAM, 8>(delta, tsm, tma);
    }
    return nullptr;
}

EvalFn pick_tiled_plain(int team, int qmax, bool delta, bool tsm, bool tma) {
    switch (team) {
        case 4: return pick1<4>(qmax, delta, tsm, tma);
        case 8: return pick1<8>(qmax, delta, tsm, tma);
        case 16: return pick1<16>(qmax, delta, tsm, tma);
        case 32: return pick1<32>(qmax, delta, tsm, tma);
    }
    return nullptr;
}

}  // namespace mm
