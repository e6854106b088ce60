// Batched move evaluation (the hot path): per (move, scenario) NPV delta,
// exact feasibility flag, scenario reduction to mean - lambda*std.
//
// Work mapping.  A "team" of TEAM lanes (4, 8, 16 or 32) evaluates one move;
// a warp therefore holds 32/TEAM moves.  Lane l of a team owns scenario quads
// q = l, l + TEAM, ... (four scenarios per quad, one 16-byte load per row), so
// a team reads each moved block's value row with coalesced 128-bit loads.
// Decode and feasibility are per-move scalar work that the team's lanes do in
// lockstep (free under SIMT).  The scenario mean and variance are reduced
// with xor-shuffles inside the team, two-pass (the deviations stay in
// registers), so a structural zero (identical blocks, a no-op) is exactly 0.
//
// Per-(move, scenario) arithmetic with uniform block mass m (all workloads):
//   block b1 moves t1 -> t2 (and, for a swap, b2 moves t2 -> t1)
//   delta_s = (v1_s - v2_s) * (d_t2 - d_t1)
//           + [o1 & !o2] (Pout[t1][s] + Pin[t2][s])
//           + [o2 & !o1] (Pin[t1][s] + Pout[t2][s])
// where v2 = 0, o2 = 0 for a shift, and Pout/Pin are the NPV changes of
// removing/adding one block of ore tonnage in (t, s), built in FP64 from the
// exact integer ore tonnage (so no penalty is formed as a difference of large
// FP32 numbers).  With unequal masses a general kernel forms the penalty
// change per (move, scenario) from the integer tonnages instead.
#include "mm_internal.cuh"
#include "mm_move.cuh"

namespace mm {

struct EvalArgs {
    const int2 *moves;
    int64_t n;
    float *score;
    uint8_t *feas;
    float *mean;
    float *delta;
    const float *val;
    const uint32_t *ore;
    const uint32_t *blk;
    const uint32_t *mass;
    const float *tab;
    const float *ddt;
    const int64_t *minedT;
    const uint64_t *cap;
    const int64_t *oreT;
    const uint64_t *target;
    const double *disc;
    uint32_t *status;
    Topo tp;
    int32_t S, S_pad, W, T;
    uint32_t m_uniform;
    float lambda;
    double a, e;
};

// Neumaier-compensated accumulation: (s, c) += x.
__device__ __forceinline__ void comp_add(float &s, float &c, float x) {
    float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

// (s, c) += (s2, c2) with an error-free TwoSum of the leading parts.
__device__ __forceinline__ void comp_merge(float &s, float &c, float s2, float c2) {
    float t = s + s2;
    float bb = t - s;
    float err = (s - (t - bb)) + (s2 - bb);
    s = t;
    c = c + c2 + err;
}

template <int TEAM>
__device__ __forceinline__ float team_sum(float x) {
#pragma unroll
    for (int off = TEAM / 2; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

template <int TEAM>
__device__ __forceinline__ void team_sum_comp(float &s, float &c) {
#pragma unroll
    for (int off = TEAM / 2; off > 0; off >>= 1) {
        float s2 = __shfl_xor_sync(0xffffffffu, s, off);
        float c2 = __shfl_xor_sync(0xffffffffu, c, off);
        comp_merge(s, c, s2, c2);
    }
}

template <bool TSM>
__device__ __forceinline__ float4 ld_tab(const float *p) {
    if (TSM) return *reinterpret_cast<const float4 *>(p);
    return __ldg(reinterpret_cast<const float4 *>(p));
}

__device__ __forceinline__ float sel_bit(uint32_t bits, int j, float x) { return ((bits >> j) & 1u) ? x : 0.0f; }

// Uniform-mass evaluator.  QPL = quads per lane (compile-time upper bound).
template <int TEAM, int QPL, bool KAHAN, bool DELTA, bool TSM>
__global__ void __launch_bounds__(256) k_eval_uniform(EvalArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T1 = A.T + 1;
    float *s_tab = reinterpret_cast<float *>(smem);                       // [2][T+1][S_pad] if TSM
    const size_t tab_floats = TSM ? (size_t)2 * T1 * A.S_pad : 0;
    float *s_dd = s_tab + tab_floats;                                      // [(T+1)^2]
    size_t off = (tab_floats + (size_t)T1 * T1) * sizeof(float);
    off = (off + 15) & ~(size_t)15;
    int64_t *s_mined = reinterpret_cast<int64_t *>(smem + off);            // [T+1]
    uint64_t *s_cap = reinterpret_cast<uint64_t *>(s_mined + T1);          // [T+1]

    if (TSM) {
        const float4 *src = reinterpret_cast<const float4 *>(A.tab);
        float4 *dst = reinterpret_cast<float4 *>(s_tab);
        for (int i = threadIdx.x; i < (int)(tab_floats / 4); i += blockDim.x) dst[i] = __ldg(src + i);
    }
    for (int i = threadIdx.x; i < T1 * T1; i += blockDim.x) s_dd[i] = __ldg(A.ddt + i);
    for (int i = threadIdx.x; i < T1; i += blockDim.x) {
        s_mined[i] = A.minedT[i];
        s_cap[i] = A.cap[i];
    }
    __syncthreads();
    const float *tab = TSM ? s_tab : A.tab;

    constexpr int TPW = 32 / TEAM;
    const int lane = threadIdx.x & 31;
    const int tl = lane % TEAM;
    const int tw = lane / TEAM;
    const int64_t warp_gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int S = A.S, S_pad = A.S_pad, W = A.W;
    const int NQ = (S + 3) >> 2;
    const int rem = S - 4 * (NQ - 1);  // valid scenarios in the last quad (1..4)
    const float invS = 1.0f / (float)S;
    const size_t pin_off = (size_t)T1 * S_pad;

    for (int64_t base = warp_gid * TPW; base < A.n; base += nwarps * TPW) {
        const int64_t i = base + tw;
        const bool active = i < A.n;
        const int2 mv = active ? __ldg(A.moves + i) : make_int2(0, -1);
        const MoveView v = decode_move(
            mv, A.tp, [&](int32_t b) { return __ldg(A.blk + b); }, [&](int32_t) { return A.m_uniform; },
            [&](uint32_t t) { return s_mined[t]; }, [&](uint32_t t) { return s_cap[t]; });
        const bool work = active && v.valid && !v.noop;
        const bool sw = v.swap;
        const int32_t b1 = work ? v.b1 : 0;
        const int32_t b2 = (work && sw) ? v.b2 : 0;
        const uint32_t t1 = work ? v.t1 : 0, t2 = work ? v.t2 : 0;
        const float dd = s_dd[t1 * T1 + t2];
        const float4 *r1 = reinterpret_cast<const float4 *>(A.val + (int64_t)b1 * S_pad);
        const float4 *r2 = reinterpret_cast<const float4 *>(A.val + (int64_t)b2 * S_pad);
        const uint32_t *o1w = A.ore + (int64_t)b1 * W;
        const uint32_t *o2w = A.ore + (int64_t)b2 * W;
        const float *pout1 = tab + (size_t)t1 * S_pad;
        const float *pin2 = tab + pin_off + (size_t)t2 * S_pad;
        const float *pin1 = tab + pin_off + (size_t)t1 * S_pad;
        const float *pout2 = tab + (size_t)t2 * S_pad;

        float d[QPL][4];
        float sum = 0.0f, csum = 0.0f;
#pragma unroll
        for (int k = 0; k < QPL; k++) {
            const int q = tl + k * TEAM;
#pragma unroll
            for (int j = 0; j < 4; j++) d[k][j] = 0.0f;
            if (work && q < NQ) {
                const float4 a = __ldg(r1 + q);
                const uint32_t n1 = (__ldg(o1w + (q >> 3)) >> ((q & 7) * 4)) & 0xfu;
                float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
                uint32_t n2 = 0;
                if (sw) {
                    b = __ldg(r2 + q);
                    n2 = (__ldg(o2w + (q >> 3)) >> ((q & 7) * 4)) & 0xfu;
                }
                const uint32_t g1 = n1 & ~n2, g2 = n2 & ~n1;
                const float4 pa = ld_tab<TSM>(pout1 + 4 * q);
                const float4 pb = ld_tab<TSM>(pin2 + 4 * q);
                float4 pc = make_float4(0.f, 0.f, 0.f, 0.f), pd = pc;
                if (sw) {
                    pc = ld_tab<TSM>(pin1 + 4 * q);
                    pd = ld_tab<TSM>(pout2 + 4 * q);
                }
                d[k][0] = fmaf(a.x - b.x, dd, sel_bit(g1, 0, pa.x + pb.x) + sel_bit(g2, 0, pc.x + pd.x));
                d[k][1] = fmaf(a.y - b.y, dd, sel_bit(g1, 1, pa.y + pb.y) + sel_bit(g2, 1, pc.y + pd.y));
                d[k][2] = fmaf(a.z - b.z, dd, sel_bit(g1, 2, pa.z + pb.z) + sel_bit(g2, 2, pc.z + pd.z));
                d[k][3] = fmaf(a.w - b.w, dd, sel_bit(g1, 3, pa.w + pb.w) + sel_bit(g2, 3, pc.w + pd.w));
                // padding scenarios have zero rows and zero ore bits: d = 0 there
            }
            if (KAHAN) {
#pragma unroll
                for (int j = 0; j < 4; j++) comp_add(sum, csum, d[k][j]);
            } else {
                sum += (d[k][0] + d[k][1]) + (d[k][2] + d[k][3]);
            }
        }
        float mu;
        if (KAHAN) {
            team_sum_comp<TEAM>(sum, csum);
            mu = (sum + csum) * invS;
        } else {
            mu = team_sum<TEAM>(sum) * invS;
        }
        float var = 0.0f, cvar = 0.0f;
#pragma unroll
        for (int k = 0; k < QPL; k++) {
            const int q = tl + k * TEAM;
            if (q < NQ) {
                const int nv = (q == NQ - 1) ? rem : 4;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const float dv = (j < nv) ? d[k][j] - mu : 0.0f;
                    if (KAHAN) comp_add(var, cvar, dv * dv);
                    else var = fmaf(dv, dv, var);
                }
            }
        }
        if (KAHAN) {
            team_sum_comp<TEAM>(var, cvar);
            var = var + cvar;
        } else {
            var = team_sum<TEAM>(var);
        }
        const float sd = sqrtf(var * invS);
        if (active) {
            if (tl == 0) {
                float sc, mn;
                if (!v.valid) {
                    sc = -INFINITY;
                    mn = 0.0f;
                    atomicOr(A.status, kStBadMove);
                } else if (!work) {
                    sc = 0.0f;
                    mn = 0.0f;
                } else {
                    sc = mu - A.lambda * sd;
                    mn = mu;
                }
                A.score[i] = sc;
                A.feas[i] = v.feasible ? 1 : 0;
                if (A.mean) A.mean[i] = mn;
            }
            if (DELTA) {
                float *drow = A.delta + i * (int64_t)S;
#pragma unroll
                for (int k = 0; k < QPL; k++) {
                    const int q = tl + k * TEAM;
                    if (q < NQ) {
                        const int nv = (q == NQ - 1) ? rem : 4;
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            if (j < nv) drow[4 * q + j] = d[k][j];
                    }
                }
            }
        }
    }
}

// General evaluator (unequal block masses): one warp per move, one lane per
// scenario, penalty change from the exact integer ore tonnages:
//   dO = m2*o2 - m1*o1 enters period t1 and leaves period t2;
//   delta_s = (v1 - v2)(d_t2 - d_t1) + d_t1 (pen(x1) - pen(x1 + dO)) + d_t2 (pen(x2) - pen(x2 - dO)).
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
    const int S = A.S, S_pad = A.S_pad, W = A.W, T1 = A.T + 1;
    for (int64_t i = warp_gid; i < A.n; i += nwarps) {
        const int2 mv = __ldg(A.moves + i);
        const MoveView v = decode_move(
            mv, A.tp, [&](int32_t b) { return __ldg(A.blk + b); }, [&](int32_t b) { return __ldg(A.mass + b); },
            [&](uint32_t t) { return A.minedT[t]; }, [&](uint32_t t) { return A.cap[t]; });
        const bool work = v.valid && !v.noop;
        float sum = 0.0f;
        float dl[kMaxS / 32];
        const float dd = work ? __ldg(A.ddt + v.t1 * T1 + v.t2) : 0.0f;
#pragma unroll 4
        for (int k = 0; k < kMaxS / 32; k++) {
            const int s = lane + 32 * k;
            float x = 0.0f;
            if (work && s < S) {
                const uint32_t o1 = (__ldg(A.ore + (int64_t)v.b1 * W + (s >> 5)) >> (s & 31)) & 1u;
                const float v1 = __ldg(A.val + (int64_t)v.b1 * S_pad + s);
                uint32_t o2 = 0;
                float v2 = 0.0f;
                if (v.swap) {
                    o2 = (__ldg(A.ore + (int64_t)v.b2 * W + (s >> 5)) >> (s & 31)) & 1u;
                    v2 = __ldg(A.val + (int64_t)v.b2 * S_pad + s);
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
                x = fmaf(v1 - v2, dd, (float)p);
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

using EvalFn = void (*)(EvalArgs);

template <int TEAM, int QPL, bool TSM>
static EvalFn pick_uniform(bool kahan, bool delta) {
    if (kahan) return delta ? k_eval_uniform<TEAM, QPL, true, true, TSM> : k_eval_uniform<TEAM, QPL, true, false, TSM>;
    return delta ? k_eval_uniform<TEAM, QPL, false, true, TSM> : k_eval_uniform<TEAM, QPL, false, false, TSM>;
}

template <int TEAM, bool TSM>
static EvalFn pick_qpl(int qpl, bool kahan, bool delta) {
    if (qpl <= 1) return pick_uniform<TEAM, 1, TSM>(kahan, delta);
    if (qpl <= 2) return pick_uniform<TEAM, 2, TSM>(kahan, delta);
    if (qpl <= 4) return pick_uniform<TEAM, 4, TSM>(kahan, delta);
    if (qpl <= 8) return pick_uniform<TEAM, 8, TSM>(kahan, delta);
    return nullptr;
}

template <bool TSM>
static EvalFn pick_team(int team, int qpl, bool kahan, bool delta) {
    switch (team) {
        case 4: return pick_qpl<4, TSM>(qpl, kahan, delta);
        case 8: return pick_qpl<8, TSM>(qpl, kahan, delta);
        case 16: return pick_qpl<16, TSM>(qpl, kahan, delta);
        case 32: return pick_qpl<32, TSM>(qpl, kahan, delta);
    }
    return nullptr;
}

// Team size: smallest power of two in 4..32 that keeps quads per lane <= 4,
// else 32 lanes with up to 8 quads per lane.
int default_team(int S) {
    int nq = (S + 3) / 4;
    for (int team = 4; team <= 32; team *= 2)
        if ((nq + team - 1) / team <= 4) return team;
    return 32;
}

mm_status eval_launch(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas, float *mean,
                      float *delta, int32_t options, int team, int ctas_per_sm) {
    EvalArgs A;
    A.moves = reinterpret_cast<const int2 *>(moves);
    A.n = n;
    A.score = score; A.feas = feas; A.mean = mean; A.delta = delta;
    A.val = m->val; A.ore = m->ore; A.blk = m->blk; A.mass = m->mass;
    A.tab = m->tab; A.ddt = m->ddt; A.minedT = m->minedT; A.cap = m->cap;
    A.oreT = m->oreT; A.target = m->target; A.disc = m->disc;
    A.status = m->status;
    A.tp.B = m->B; A.tp.T = m->T; A.tp.nx = m->nx; A.tp.ny = m->ny; A.tp.nz = m->nz;
    A.tp.pred_ptr = m->pred_ptr; A.tp.pred_idx = m->pred_idx; A.tp.succ_ptr = m->succ_ptr; A.tp.succ_idx = m->succ_idx;
    A.S = m->S; A.S_pad = m->S_pad; A.W = m->W; A.T = m->T;
    A.m_uniform = m->m_uniform;
    A.lambda = (float)m->lambda;
    A.a = m->shortfall_pen; A.e = m->excess_pen;
    const bool kahan = (options & MM_EVAL_KAHAN) != 0;
    const bool want_delta = delta != nullptr;
    const int threads = 256;
    if (!m->uniform_mass) {
        EvalFn fn = want_delta ? k_eval_general<true> : k_eval_general<false>;
        int64_t warps_needed = n;
        int64_t blocks = (warps_needed + 7) / 8;
        int64_t cap_blocks = (int64_t)m->num_sms * 8;
        if (blocks > cap_blocks) blocks = cap_blocks;
        if (blocks < 1) blocks = 1;
        fn<<<(unsigned)blocks, threads, 0, m->stream>>>(A);
        return check_launch("k_eval_general");
    }
    if (team <= 0) team = default_team(m->S);
    const int nq = (m->S + 3) / 4;
    const int qpl = (nq + team - 1) / team;
    const int T1 = m->T + 1;
    const size_t tab_bytes = (size_t)2 * T1 * m->S_pad * sizeof(float);
    const size_t small = (((size_t)T1 * T1 * sizeof(float) + 15) & ~(size_t)15) + 2 * (size_t)T1 * sizeof(int64_t);
    const bool tsm = tab_bytes <= 48 * 1024;
    const size_t smem = (tsm ? tab_bytes : 0) + small;
    EvalFn fn = tsm ? pick_team<true>(team, qpl, kahan, want_delta) : pick_team<false>(team, qpl, kahan, want_delta);
    if (!fn) return set_error(MM_ERR_INVALID_ARG, "no evaluator for team %d with %d quads per lane", team, qpl);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e, "set evaluator shared memory");
    }
    int per_sm = ctas_per_sm;
    if (per_sm <= 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
        if (e != cudaSuccess) return cuda_status(e, "occupancy query");
        if (per_sm < 1) per_sm = 1;
    }
    const int64_t moves_per_cta = (int64_t)(threads / 32) * (32 / team);
    int64_t blocks = (n + moves_per_cta - 1) / moves_per_cta;
    const int64_t grid_cap = (int64_t)m->num_sms * per_sm;
    if (blocks > grid_cap) blocks = grid_cap;
    if (blocks < 1) blocks = 1;
    fn<<<(unsigned)blocks, threads, smem, m->stream>>>(A);
    return check_launch("k_eval_uniform");
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
    return eval_launch(m, moves, n, score, feas, mean, nullptr, MM_EVAL_PLAIN, m->team, m->ctas_per_sm);
}

mm_status mm_set_tile(mm_model *m, int32_t team, int32_t ctas_per_sm) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (team != 0 && team != 4 && team != 8 && team != 16 && team != 32)
        return set_error(MM_ERR_INVALID_ARG, "team must be 0, 4, 8, 16 or 32");
    if (team != 0 && ((m->S + 3) / 4 + team - 1) / team > 8)
        return set_error(MM_ERR_INVALID_ARG, "team %d leaves more than 8 quads per lane at S = %d", team, m->S);
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return set_error(MM_ERR_INVALID_ARG, "ctas_per_sm out of range");
    m->team = team;
    m->ctas_per_sm = ctas_per_sm;
    return MM_OK;
}

mm_status mm_eval_moves_ex(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas, float *mean,
                           float *delta, int32_t options) {
    mm_status st = eval_check(m, moves, n, score, feas);
    if (st != MM_OK || n == 0) return st;
    if (options & ~MM_EVAL_KAHAN) return set_error(MM_ERR_INVALID_ARG, "unknown option bits 0x%x", options);
    return eval_launch(m, moves, n, score, feas, mean, delta, options, m->team, m->ctas_per_sm);
}

}  // extern "C"
