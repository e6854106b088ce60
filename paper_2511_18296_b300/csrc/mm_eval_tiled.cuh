// Tiled move evaluator (the hot kernel), uniform block mass.
//
// Every warp of the persistent grid owns a contiguous, equal share of the
// batch and walks it in chunks of 64 moves:
//   1. decode   two moves per lane: bounds check, exact feasibility flag
//               (packed lo/hi schedule words, shared-memory tonnage), no-op
//               detection; the flag is stored at once; working moves are
//               appended to a shift list or a swap list (warp ballots);
//   2. compute  teams of TEAM lanes take list entries, so every team runs a
//               branch-free loop specialised for its move type: a shift reads
//               one value row and two penalty-table rows, a swap two value
//               rows and four table rows (a shift never does a swap's work);
//   3. store    scores/means staged in shared memory go out coalesced.
// Warps never wait on each other (no CTA barrier after the table staging).
// The next chunk's moves are loaded into registers while the current chunk is
// processed.  Per scenario quad a lane issues one 16-byte row load per moved
// block, one ore word (shared by 8 lanes) and 16-byte table loads from shared
// memory; ore bits become 0/1 float masks through a 16-entry table, so the
// per-scenario work is four (shift) or seven (swap) FP32 operations.
#pragma once

#include "mm_internal.cuh"
#include "mm_move.cuh"

namespace mm {

#ifndef MM_EVAL_MINB
#define MM_EVAL_MINB 3  // minimum resident CTAs per SM requested from the register allocator
#endif

constexpr int kEvalThreads = 256;  // threads per CTA
constexpr int kChunk = 64;         // moves a warp decodes at once (two per lane)

struct EvalArgs {
    const int2 *moves;
    int64_t n;
    float *score;
    uint8_t *feas;
    float *mean;
    float *delta;
    const float *val;      // [B+1][S_pad], row B = zeros (stand-in partner of a shift)
    const uint32_t *ore;   // [B+1][W],     row B = zeros
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
    int32_t qpl;           // quads per lane actually used (<= QMAX)
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

// Ore bits of quad q (scenarios 4q..4q+3) of an ore row.
template <int TEAM>
__device__ __forceinline__ uint32_t ore_nibble(const uint32_t *orow, int q) {
    return (__ldg(orow + (q >> 3)) >> ((q & 7) * 4)) & 0xfu;
}

// Per-move scenario loop + reduction for one team.  SWAP selects the move
// type at compile time.  Returns the mean; writes the deltas to d[][].
template <int TEAM, int QMAX, bool SWAP, bool KAHAN>
__device__ __forceinline__ void team_eval(const EvalArgs &A, const float *tab, const float4 *lut, int tl, bool act,
                                          int32_t b1, int32_t b2, uint32_t t1, uint32_t t2, float dd, int NQ,
                                          int rem, float invS, size_t pin_off, float (&d)[QMAX][4], float &mu,
                                          float &sd) {
    const int S_pad = A.S_pad, W = A.W;
    const float *vrow1 = A.val + (size_t)b1 * S_pad;
    const float *vrow2 = A.val + (size_t)b2 * S_pad;
    const uint32_t *orow1 = A.ore + (size_t)b1 * W;
    const uint32_t *orow2 = A.ore + (size_t)b2 * W;
    const int pout1 = (int)t1 * S_pad, pout2 = (int)t2 * S_pad;
    const int pin1 = (int)pin_off + pout1, pin2 = (int)pin_off + pout2;
    const int nq = act ? NQ : 0;
    float sum = 0.0f, csum = 0.0f;
#pragma unroll
    for (int k = 0; k < QMAX; k++) {
        const int q = tl + k * TEAM;
#pragma unroll
        for (int j = 0; j < 4; j++) d[k][j] = 0.0f;
        if (k < A.qpl && q < nq) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(vrow1) + q);
            const float4 pa = ld_tab<true>(tab + pout1 + 4 * q);
            const float4 pb = ld_tab<true>(tab + pin2 + 4 * q);
            if (SWAP) {
                const float4 b = __ldg(reinterpret_cast<const float4 *>(vrow2) + q);
                const uint32_t n1 = ore_nibble<TEAM>(orow1, q);
                const uint32_t n2 = ore_nibble<TEAM>(orow2, q);
                const float4 m1 = lut[n1 & ~n2];
                const float4 m2 = lut[n2 & ~n1];
                const float4 pc = ld_tab<true>(tab + pin1 + 4 * q);
                const float4 pd = ld_tab<true>(tab + pout2 + 4 * q);
                d[k][0] = fmaf(a.x - b.x, dd, fmaf(m2.x, pc.x + pd.x, m1.x * (pa.x + pb.x)));
                d[k][1] = fmaf(a.y - b.y, dd, fmaf(m2.y, pc.y + pd.y, m1.y * (pa.y + pb.y)));
                d[k][2] = fmaf(a.z - b.z, dd, fmaf(m2.z, pc.z + pd.z, m1.z * (pa.z + pb.z)));
                d[k][3] = fmaf(a.w - b.w, dd, fmaf(m2.w, pc.w + pd.w, m1.w * (pa.w + pb.w)));
            } else {
                const float4 m1 = lut[ore_nibble<TEAM>(orow1, q)];
                d[k][0] = fmaf(a.x, dd, m1.x * (pa.x + pb.x));
                d[k][1] = fmaf(a.y, dd, m1.y * (pa.y + pb.y));
                d[k][2] = fmaf(a.z, dd, m1.z * (pa.z + pb.z));
                d[k][3] = fmaf(a.w, dd, m1.w * (pa.w + pb.w));
            }
            // padding scenarios (s >= S) have zero rows and zero ore bits: d = 0 there
        }
        if (KAHAN) {
#pragma unroll
            for (int j = 0; j < 4; j++) comp_add(sum, csum, d[k][j]);
        } else {
            sum += (d[k][0] + d[k][1]) + (d[k][2] + d[k][3]);
        }
    }
    if (KAHAN) {
        team_sum_comp<TEAM>(sum, csum);
        mu = (sum + csum) * invS;
    } else {
        mu = team_sum<TEAM>(sum) * invS;
    }
    float var = 0.0f, cvar = 0.0f;
#pragma unroll
    for (int k = 0; k < QMAX; k++) {
        const int q = tl + k * TEAM;
        if (k < A.qpl && q < nq) {
            float dv[4];
#pragma unroll
            for (int j = 0; j < 4; j++) dv[j] = d[k][j] - mu;
            if (rem != 4 && q == NQ - 1) {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (j >= rem) dv[j] = 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (KAHAN) comp_add(var, cvar, dv[j] * dv[j]);
                else var = fmaf(dv[j], dv[j], var);
            }
        }
    }
    if (KAHAN) {
        team_sum_comp<TEAM>(var, cvar);
        var = var + cvar;
    } else {
        var = team_sum<TEAM>(var);
    }
    sd = sqrtf(var * invS);
}

template <int TEAM, int QMAX, bool KAHAN, bool DELTA, bool TSM>
__global__ void __launch_bounds__(kEvalThreads, MM_EVAL_MINB) k_eval_tiled(EvalArgs A) {
    constexpr int CH = kChunk;              // moves per warp chunk (2 per lane)
    constexpr int NW = kEvalThreads / 32;   // warps per CTA
    constexpr int TPW = 32 / TEAM;          // teams per warp
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float4 s_lut[16];
    __shared__ int32_t s_b1[NW][CH], s_b2[NW][CH];
    __shared__ uint32_t s_tt[NW][CH];
    __shared__ uint8_t s_lsh[NW][CH], s_lsw[NW][CH];
    __shared__ float s_score[NW][CH], s_mean[NW][CH];

    const int T1 = A.T + 1;
    const size_t tab_floats = (size_t)2 * T1 * A.S_pad;
    float *s_tab = reinterpret_cast<float *>(smem);                            // [2][T+1][S_pad] if TSM
    float *s_dd = s_tab + (TSM ? tab_floats : 0);                              // [(T+1)^2]
    size_t off = ((TSM ? tab_floats : 0) + (size_t)T1 * T1) * sizeof(float);
    off = (off + 15) & ~(size_t)15;
    int64_t *s_mined = reinterpret_cast<int64_t *>(smem + off);                // [T+1]
    uint64_t *s_cap = reinterpret_cast<uint64_t *>(s_mined + T1);              // [T+1]

    const int tid = threadIdx.x;
    if (TSM) {
        const float4 *src = reinterpret_cast<const float4 *>(A.tab);
        float4 *dst = reinterpret_cast<float4 *>(s_tab);
        for (int i = tid; i < (int)(tab_floats / 4); i += kEvalThreads) dst[i] = __ldg(src + i);
    }
    for (int i = tid; i < T1 * T1; i += kEvalThreads) s_dd[i] = __ldg(A.ddt + i);
    for (int i = tid; i < T1; i += kEvalThreads) {
        s_mined[i] = A.minedT[i];
        s_cap[i] = A.cap[i];
    }
    if (tid < 16)
        s_lut[tid] = make_float4((float)(tid & 1), (float)((tid >> 1) & 1), (float)((tid >> 2) & 1),
                                 (float)((tid >> 3) & 1));
    __syncthreads();
    const float *tab = TSM ? s_tab : A.tab;

    const int lane = tid & 31, warp = tid >> 5;
    const int tl = lane % TEAM, tw = lane / TEAM;
    const int S = A.S;
    const int NQ = (S + 3) >> 2;
    const int rem = S - 4 * (NQ - 1);
    const float invS = 1.0f / (float)S;
    const size_t pin_off = (size_t)T1 * A.S_pad;
    const uint32_t lt_mask = (1u << lane) - 1u;
    // contiguous, balanced range of moves for this warp
    const int64_t nwarps = (int64_t)gridDim.x * NW;
    const int64_t gw = (int64_t)blockIdx.x * NW + warp;
    const int64_t r0 = gw * A.n / nwarps, r1 = (gw + 1) * A.n / nwarps;

    int2 mv[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int64_t i = r0 + h * 32 + lane;
        mv[h] = i < r1 ? __ldg(A.moves + i) : make_int2(0, -1);
    }
    for (int64_t c0 = r0; c0 < r1; c0 += CH) {
        // ---- decode: two moves per lane ----
        int nsh = 0, nsw = 0;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int slot = h * 32 + lane;
            const int64_t i = c0 + slot;
            const bool active = i < r1;
            const MoveView v = decode_move(
                mv[h], A.tp, [&](int32_t b) { return __ldg(A.blk + b); }, [&](int32_t) { return A.m_uniform; },
                [&](uint32_t t) { return s_mined[t]; }, [&](uint32_t t) { return s_cap[t]; });
            const int64_t ni = i + CH;  // prefetch the next chunk's move
            mv[h] = ni < r1 ? __ldg(A.moves + ni) : make_int2(0, -1);
            const bool work = active && v.valid && !v.noop;
            if (active) {
                A.feas[i] = v.feasible ? 1 : 0;
                if (!v.valid) atomicOr(A.status, kStBadMove);
                if (DELTA && !work) {
                    float *drow = A.delta + i * (int64_t)S;
                    for (int s2 = 0; s2 < S; s2++) drow[s2] = 0.0f;
                }
            }
            s_score[warp][slot] = v.valid ? 0.0f : -INFINITY;
            s_mean[warp][slot] = 0.0f;
            if (work) {
                s_b1[warp][slot] = v.b1;
                s_b2[warp][slot] = v.swap ? v.b2 : A.tp.B;
                s_tt[warp][slot] = v.t1 | (v.t2 << 8);
            }
            const bool is_sh = work && !v.swap, is_sw = work && v.swap;
            const uint32_t msh = __ballot_sync(0xffffffffu, is_sh);
            const uint32_t msw = __ballot_sync(0xffffffffu, is_sw);
            if (is_sh) s_lsh[warp][nsh + __popc(msh & lt_mask)] = (uint8_t)slot;
            if (is_sw) s_lsw[warp][nsw + __popc(msw & lt_mask)] = (uint8_t)slot;
            nsh += __popc(msh);
            nsw += __popc(msw);
        }
        __syncwarp();
        // ---- compute: teams over the shift list, then the swap list ----
#pragma unroll 1
        for (int pass = 0; pass < 2; pass++) {
            const int nl = pass == 0 ? nsh : nsw;
            const uint8_t *list = pass == 0 ? s_lsh[warp] : s_lsw[warp];
#pragma unroll 1
            for (int eb = 0; eb < nl; eb += TPW) {
                const int e = eb + tw;
                const bool act = e < nl;
                const int slot = act ? list[e] : 0;
                const int32_t b1 = act ? s_b1[warp][slot] : 0;
                const int32_t b2 = act ? s_b2[warp][slot] : 0;
                const uint32_t tt = act ? s_tt[warp][slot] : 0;
                const uint32_t t1 = tt & 0xffu, t2 = tt >> 8;
                const float dd = s_dd[t1 * T1 + t2];
                float d[QMAX][4];
                float mu, sd;
                if (pass == 0)
                    team_eval<TEAM, QMAX, false, KAHAN>(A, tab, s_lut, tl, act, b1, b2, t1, t2, dd, NQ, rem, invS,
                                                        pin_off, d, mu, sd);
                else
                    team_eval<TEAM, QMAX, true, KAHAN>(A, tab, s_lut, tl, act, b1, b2, t1, t2, dd, NQ, rem, invS,
                                                       pin_off, d, mu, sd);
                if (act) {
                    if (tl == 0) {
                        s_score[warp][slot] = mu - A.lambda * sd;
                        s_mean[warp][slot] = mu;
                    }
                    if (DELTA) {
                        float *drow = A.delta + (c0 + slot) * (int64_t)S;
#pragma unroll
                        for (int k = 0; k < QMAX; k++) {
                            const int q = tl + k * TEAM;
                            if (k < A.qpl && q < NQ) {
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
        __syncwarp();
        // ---- store (coalesced) ----
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int slot = h * 32 + lane;
            const int64_t i = c0 + slot;
            if (i < r1) {
                A.score[i] = s_score[warp][slot];
                if (A.mean) A.mean[i] = s_mean[warp][slot];
            }
        }
        __syncwarp();
    }
}

}  // namespace mm
