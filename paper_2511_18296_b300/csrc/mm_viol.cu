// Violation magnitudes of candidate moves, for the epsilon-relaxed fitness of
// the paper's search (Algorithm 2: fitness = NPV - penalty max(0, violation -
// epsilon); Section 6 Phase 2: ... - gamma max(0, violation - epsilon(t))).
// The paper does not define violation(S) beyond "constraint violation"; for a
// move x -> x' this library reports two exact integers that are both zero
// exactly when the move's feasibility flag is 1:
//   capacity excess  = sum over the distinct periods t < T that a moved block
//                      leaves or enters of max(0, mined'_t - M_t)   (tonnes)
//   precedence excess = sum over the moved blocks b of
//                      max(0, L_b - x'_b) + max(0, x'_b - H_b)     (periods)
//     with L_b the latest predecessor period and H_b the earliest successor
//     period in x' (0 and T when there are none): how far b would have to move
//     to satisfy every arc at it (Eq. 15).
// One thread per move; the packed lo/hi word gives L_b and H_b except when a
// swap's two blocks are direct neighbours, where the bounds are re-read from
// the neighbours' periods with the partner's new period.
#include "mm_apply.cuh"

namespace mm {

Topo topo_of_model(const mm_model *m);

struct ViolArgs {
    const int2 *moves;
    int64_t n;
    int64_t *cap_excess;
    int32_t *prec_excess;
    const uint32_t *blk;
    const uint32_t *mass;
    const int64_t *minedT;
    const uint64_t *cap;
    Topo tp;
    uint32_t m_uniform;
    int32_t uniform;
    uint32_t *status;
};

// L_b and H_b of block b in x' where the only other moved block is p (new
// period tp): neighbours' periods read one by one (grid pattern or CSR).
__device__ __forceinline__ void bounds_with_partner(const ViolArgs &A, int32_t b, int32_t p, uint32_t tp,
                                                    uint32_t &L, uint32_t &H) {
    auto period = [&](int32_t j) -> uint32_t { return j == p ? tp : blk_period(__ldg(A.blk + j)); };
    const uint32_t w = block_bounds(A.tp, b, period);
    L = blk_lo(w);
    H = blk_hi(w);
}

__device__ __forceinline__ int64_t excess_of(int64_t mined, uint64_t cap) {
    return mined > (int64_t)cap ? mined - (int64_t)cap : 0;
}

__device__ __forceinline__ int32_t outside(uint32_t t, uint32_t L, uint32_t H) {
    return (int32_t)(L > t ? L - t : 0u) + (int32_t)(t > H ? t - H : 0u);
}

__global__ void __launch_bounds__(256) k_violation(ViolArgs A) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint32_t T = (uint32_t)A.tp.T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride) {
        const int2 mv = __ldg(A.moves + i);
        const bool swap = mv.y >= 0;
        const int64_t tn = -(int64_t)mv.y - 1;
        const bool valid = mv.x >= 0 && mv.x < A.tp.B && (swap ? mv.y < A.tp.B : (tn >= 0 && tn <= (int64_t)T));
        if (!valid) {
            A.cap_excess[i] = -1;
            A.prec_excess[i] = -1;
            atomicOr(A.status, kStBadMove);
            continue;
        }
        const int32_t b1 = mv.x, b2 = swap ? mv.y : -1;
        const uint32_t w1 = __ldg(A.blk + b1);
        const uint32_t w2 = swap ? __ldg(A.blk + b2) : 0u;
        const uint32_t t1 = blk_period(w1), t2 = swap ? blk_period(w2) : (uint32_t)tn;
        const int64_t m1 = A.uniform ? (int64_t)A.m_uniform : (int64_t)__ldg(A.mass + b1);
        const int64_t m2 = swap ? (A.uniform ? (int64_t)A.m_uniform : (int64_t)__ldg(A.mass + b2)) : 0;
        // capacity: the distinct periods left or entered (a no-op touches t1 only)
        int64_t ce = 0;
        if (t1 == t2 || (swap && b1 == b2)) {
            if (t1 < T) ce = excess_of(A.minedT[t1], A.cap[t1]);
        } else {
            if (t1 < T) ce += excess_of(A.minedT[t1] - m1 + m2, A.cap[t1]);
            if (t2 < T) ce += excess_of(A.minedT[t2] + m1 - m2, A.cap[t2]);
        }
        // precedence: b1 now in t2 (and b2 in t1)
        int32_t pe;
        if (!swap || b1 == b2) {
            pe = outside(t2, blk_lo(w1), blk_hi(w1));
        } else if (is_pred(A.tp, b2, b1) || is_pred(A.tp, b1, b2)) {
            uint32_t L, H;
            bounds_with_partner(A, b1, b2, t1, L, H);
            pe = outside(t2, L, H);
            bounds_with_partner(A, b2, b1, t2, L, H);
            pe += outside(t1, L, H);
        } else {
            pe = outside(t2, blk_lo(w1), blk_hi(w1)) + outside(t1, blk_lo(w2), blk_hi(w2));
        }
        A.cap_excess[i] = ce;
        A.prec_excess[i] = pe;
    }
}

}  // namespace mm

using namespace mm;

extern "C" mm_status mm_eval_violation(mm_model *m, const mm_move *moves, int64_t n, int64_t *cap_excess,
                                       int32_t *prec_excess) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    if (n < 0) return set_error(MM_ERR_INVALID_ARG, "negative move count");
    if (n == 0) return MM_OK;
    if (!moves || !cap_excess || !prec_excess) return set_error(MM_ERR_INVALID_ARG, "NULL output or move pointer");
    if (((uintptr_t)moves & 7u) != 0) return set_error(MM_ERR_INVALID_ARG, "moves must be 8-byte aligned");
    ViolArgs A;
    A.moves = reinterpret_cast<const int2 *>(moves);
    A.n = n;
    A.cap_excess = cap_excess;
    A.prec_excess = prec_excess;
    A.blk = m->blk;
    A.mass = m->mass;
    A.minedT = m->minedT;
    A.cap = m->cap;
    A.tp = topo_of_model(m);
    A.m_uniform = m->m_uniform;
    A.uniform = m->uniform_mass;
    A.status = m->status;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)m->num_sms * 8) blocks = (int64_t)m->num_sms * 8;
    k_violation<<<(unsigned)blocks, 256, 0, m->stream>>>(A);
    return check_launch("k_violation");
}
