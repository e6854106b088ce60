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
// block and 16-byte period-pair table loads; the ore words of a row come with
// one 16-byte load per lane where they fit (else one word per quad), and ore
// bits become 0/1 float masks by selects (the L1 data path, not the ALUs,
// limits this kernel, so a shared-memory lookup table costs more), so the
// per-scenario work is four (shift) or seven (swap) FP32 operations.
#pragma once

#include <type_traits>

#include "mm_apply.cuh"
#include "mm_sort.cuh"

namespace mm {

#ifndef MM_EVAL_MINB
#define MM_EVAL_MINB 3  // minimum resident CTAs per SM requested from the register allocator
#endif

constexpr int kEvalThreads = 256;  // threads per CTA
constexpr int kStepThreads = 768;  // threads per CTA of the fused search step: one CTA per SM, so the
                                   // batch's top-k lists (one per CTA) meet in a single level
constexpr int kChunk = 64;         // moves a warp decodes at once (two per lane)

// Where a batch's top-k lists meet: the per-CTA lists, the merged lists of
// groups of CTAs and the tickets that pick the merging CTAs.
struct StepLists {
    uint64_t *cta;        // [grid][32] each CTA's 32 best keys
    uint64_t *grp;        // [groups][32] each group's 32 best keys
    int4 *cinf, *ginf;    // [grid], [groups] the move of each list's best key: (b1, b2 or B, t1 | t2 << 8, 0)
    uint32_t *tick;       // [groups] group tickets; tick[final_slot] the final ticket
    int32_t final_slot;
    int32_t grp_size;     // CTAs per group (the last group may be smaller)
};

// What the end of a top-k launch needs (step_reduce): the lists, the
// outputs, and for an in-launch apply of the best move the batch and the
// model's apply arguments.
struct StepTail {
    StepLists L;
    int32_t k;             // top-k size, 1..32
    int64_t n;             // moves in the batch
    uint32_t *status;      // sticky status bits
    int32_t *idx_out;      // [k]
    float *top_out;        // [k]
    int32_t *count_out;    // [1]
    int32_t do_apply;      // the final CTA applies the best move (S <= CTA threads)
    const int2 *moves;     // the batch (do_apply)
    ApplyArgs ap;          // the model's apply arguments (fused step)
    int4 *pending;         // fused step: the move whose FP64 update is still due, (b1, b2 or B,
                           // t1 | t2 << 8, due); the next step's CTAs do it, a share of the scenarios each
};

struct EvalArgs {
    const int2 *moves;
    const uint32_t *pmoves;  // the batch in the compact 4-byte form instead (fused step), else nullptr
    int64_t n;
    float *score;
    uint8_t *feas;
    float *mean;
    float *delta;
    const float *val;      // [B+1][R] combined rows (values, then ore words), row B = zeros
    const uint32_t *blk;
    const uint32_t *mass;
    const float *tab;
    const float *ctab;  // [T+1][T+1][S_pad] Pout[a] + Pin[b] (the fast form reads only this)
    const float *ddt;
    const int64_t *minedT;
    const uint64_t *cap;
    const int64_t *oreT;
    const uint64_t *target;
    const double *disc;
    const float *dwt;      // [T+1][T+1][S_pad] sigma(s,b) d_b - sigma(s,a) d_a with uncertainty weights, else nullptr
    uint32_t *status;
    Topo tp;
    int32_t S, S_pad, W, T, R, ore_off;
    uint32_t m_uniform;
    int32_t qpl;           // quads per lane actually used (<= QMAX)
    int32_t nstage;        // bulk-copy pipeline depth per warp (TMA path)
    uint32_t tx_extra;     // TMA path: bytes each stage expects beyond what it copies (0; the test-only stall
                           // mode expects more, so the stage's bounded wait runs out)
    long long wait_cycles; // TMA path: limit of a stage's wait (clock cycles)
    int32_t prefetch;      // direct-load path: batches whose rows are prefetched into L1 ahead
    int32_t dd_smem;       // the (T+1)^2 discount differences are staged in shared memory (else read from ddt)
    float lambda;
    float mcm;             // mining cost of one block, mc * m (uniform mass; weighted form)
    double a, e, mc;
    StepTail tail;         // fused search step (TOPK kernels only)
};

// ---------------------------------------------------------------- warp top-k
// A warp keeps its 32 best candidate keys, one per lane, sorted best-first
// across lanes.  Keys are unique 64-bit integers: the order-preserving bits of
// the FP32 score (-0 folded into +0) above the complement of the move index,
// so larger is better and equal scores prefer the lower index; 0 = empty.

__device__ __forceinline__ uint64_t score_key(float f, int64_t i) {
    uint32_t u = __float_as_uint(f);
    if ((u << 1) == 0) u = 0;  // -0 -> +0
    const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((uint64_t)ord << 32) | (uint32_t)(~(uint32_t)i);
}

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }
__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// Bitonic sort of the 32 lane values, largest in lane 0.
__device__ __forceinline__ uint64_t warp_sort_desc(uint64_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const uint64_t y = __shfl_xor_sync(0xffffffffu, x, stride);
            const bool lower = (lane & stride) == 0;
            const bool desc = (lane & size) == 0;
            x = (lower == desc) ? umax64(x, y) : umin64(x, y);
        }
    }
    return x;
}

// Top 32 of the union of two best-first lists.
__device__ __forceinline__ uint64_t warp_merge_sorted(uint64_t t, uint64_t c) {
    const int lane = threadIdx.x & 31;
    uint64_t m = umax64(t, __shfl_sync(0xffffffffu, c, 31 - lane));  // bitonic: holds the top 32
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xffffffffu, m, stride);
        m = ((lane & stride) == 0) ? umax64(m, y) : umin64(m, y);
    }
    return m;
}

// Insert one candidate per lane (0 = none).  Candidates that beat the
// current 32nd key are inserted one by one (find the rank with a ballot,
// shift the tail of the list down one lane); more than 8 at once go through
// a full sort and merge instead.
__device__ __forceinline__ uint64_t warp_topk_insert(uint64_t t, uint64_t c) {
    const int lane = threadIdx.x & 31;
    uint32_t msk = __ballot_sync(0xffffffffu, c > __shfl_sync(0xffffffffu, t, 31));
    if (msk == 0) return t;
    if (__popc(msk) > 8) return warp_merge_sorted(t, warp_sort_desc(c));
    while (msk) {
        const int src = __ffs(msk) - 1;
        msk &= msk - 1;
        const uint64_t x = __shfl_sync(0xffffffffu, c, src);
        const int pos = __popc(__ballot_sync(0xffffffffu, t > x));  // entries better than x
        const uint64_t up = __shfl_up_sync(0xffffffffu, t, 1);
        if (pos < 32) t = lane < pos ? t : (lane == pos ? x : up);
    }
    return t;
}

// Merge another best-first list into t, skipped when it cannot contribute
// (and taken as it is when t is empty).
__device__ __forceinline__ uint64_t warp_topk_merge(uint64_t t, uint64_t c_sorted) {
    const uint64_t thr = __shfl_sync(0xffffffffu, t, 31);
    const uint64_t best = __shfl_sync(0xffffffffu, c_sorted, 0);
    if (best <= thr) return t;
    if (__shfl_sync(0xffffffffu, t, 0) == 0ull) return c_sorted;
    return warp_merge_sorted(t, c_sorted);
}


// Kahan-compensated accumulation: s += x, with c the running negative of
// the low-order part lost so far (the sum is s - c).
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
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

// Loads from a block row that lives in global memory (read-only path) or in
// shared memory (staged by a bulk copy).
template <bool SROW>
__device__ __forceinline__ float4 ld_row4(const float *row, int q) {
    if (SROW) return reinterpret_cast<const float4 *>(row)[q];
    return __ldg(reinterpret_cast<const float4 *>(row) + q);
}
template <bool SROW>
__device__ __forceinline__ uint32_t ld_ore_word(const float *row, int ore_off, int w) {
    if (SROW) return reinterpret_cast<const uint32_t *>(row + ore_off)[w];
    return __ldg(reinterpret_cast<const uint32_t *>(row + ore_off) + w);
}

// 0/1 float masks of the four bits of an ore nibble (bit j -> component j).
__device__ __forceinline__ float4 nib_mask(uint32_t n) {
    return make_float4((n & 1u) ? 1.0f : 0.0f, (n & 2u) ? 1.0f : 0.0f, (n & 4u) ? 1.0f : 0.0f,
                       (n & 8u) ? 1.0f : 0.0f);
}

// Per-move scenario loop + reduction for one team.  SWAP selects the move
// type at compile time, SROW where the two block rows live.  Writes the
// deltas to d[][], the mean to mu and the population std to sd.
template <int TEAM, int QMAX, bool SWAP, bool KAHAN, bool SROW>
__device__ __forceinline__ void team_eval(const EvalArgs &A, const float *tab, int tl, bool act,
                                          const float *row1, const float *row2, uint32_t t1, uint32_t t2, float dd,
                                          int NQ, int rem, float invS, size_t pin_off, float (&d)[QMAX][4], float &mu,
                                          float &sd) {
    const int S_pad = A.S_pad, ore_off = A.ore_off;
    const int pout1 = (int)t1 * S_pad, pout2 = (int)t2 * S_pad;
    const int pin1 = (int)pin_off + pout1, pin2 = (int)pin_off + pout2;
    const int nq = act ? NQ : 0;
    float sum = 0.0f, csum = 0.0f;
#pragma unroll
    for (int k = 0; k < QMAX; k++) {
        const int q = tl + k * TEAM;
        // loads are unconditional and in bounds (quad index clamped) so the
        // compiler can issue every quad's loads before the first use; lanes
        // past the last quad, inactive teams and k >= qpl are masked to 0.
        const int qc = q < NQ ? q : NQ - 1;
        const bool live = (k < A.qpl) && (q < nq);
        const float4 a = ld_row4<SROW>(row1, qc);
        const uint32_t sh = (qc & 7) * 4;
        const float4 pa = ld_tab<true>(tab + pout1 + 4 * qc);
        const float4 pb = ld_tab<true>(tab + pin2 + 4 * qc);
        float x[4];
        if (SWAP) {
            const float4 b = ld_row4<SROW>(row2, qc);
            const uint32_t n1 = (ld_ore_word<SROW>(row1, ore_off, qc >> 3) >> sh) & 0xfu;
            const uint32_t n2 = (ld_ore_word<SROW>(row2, ore_off, qc >> 3) >> sh) & 0xfu;
            const float4 m1 = nib_mask(n1 & ~n2);
            const float4 m2 = nib_mask(n2 & ~n1);
            const float4 pc = ld_tab<true>(tab + pin1 + 4 * qc);
            const float4 pd = ld_tab<true>(tab + pout2 + 4 * qc);
            x[0] = fmaf(a.x - b.x, dd, fmaf(m2.x, pc.x + pd.x, m1.x * (pa.x + pb.x)));
            x[1] = fmaf(a.y - b.y, dd, fmaf(m2.y, pc.y + pd.y, m1.y * (pa.y + pb.y)));
            x[2] = fmaf(a.z - b.z, dd, fmaf(m2.z, pc.z + pd.z, m1.z * (pa.z + pb.z)));
            x[3] = fmaf(a.w - b.w, dd, fmaf(m2.w, pc.w + pd.w, m1.w * (pa.w + pb.w)));
        } else {
            const float4 m1 = nib_mask((ld_ore_word<SROW>(row1, ore_off, qc >> 3) >> sh) & 0xfu);
            x[0] = fmaf(a.x, dd, m1.x * (pa.x + pb.x));
            x[1] = fmaf(a.y, dd, m1.y * (pa.y + pb.y));
            x[2] = fmaf(a.z, dd, m1.z * (pa.z + pb.z));
            x[3] = fmaf(a.w, dd, m1.w * (pa.w + pb.w));
        }
        // padding scenarios (s >= S) have zero values and zero ore bits: d = 0 there
#pragma unroll
        for (int j = 0; j < 4; j++) d[k][j] = live ? x[j] : 0.0f;
        // the fast form's order; the compensated form adds the quad's sum with Kahan's update
        if (KAHAN) kahan_add(sum, csum, (d[k][0] + d[k][2]) + (d[k][1] + d[k][3]));
        else sum += (d[k][0] + d[k][2]) + (d[k][1] + d[k][3]);
    }
    if (KAHAN) {
        csum = -csum;  // (sum, csum): the sum is sum + csum
        team_sum_comp<TEAM>(sum, csum);
        mu = (sum + csum) * invS;
    } else {
        mu = team_sum<TEAM>(sum) * invS;
    }
    float var = 0.0f;
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
            for (int j = 0; j < 4; j++) var = fmaf(dv[j], dv[j], var);
        }
    }
    var = team_sum<TEAM>(var);
    if (KAHAN) {
        // corrected two-pass variance: minus (sum of deviations)^2 / S, with
        // the deviations' sum formed as the compensated total minus S mu
        const float ds = fmaf(-(float)A.S, mu, sum) + csum;
        var = fmaxf(var - ds * ds * invS, 0.0f);
    }
    sd = sqrtf(var * invS);
}

// Two FP32 values in one 64-bit register pair and the sm_100-family paired
// instructions on them.  Each lane of fma.rn / mul.rn / add.rn / sub.rn .f32x2
// is rounded exactly like the scalar instruction, so paired and scalar code
// give the same bits; the pairing halves the issued arithmetic instructions.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t r, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Fast form of team_eval for S % 4 == 0: the team runs KF = floor(NQ / TEAM)
// full quad iterations, fixed at compile time (every lane of every team owns
// a real quad, offsets are compile-time immediates from per-lane bases, no
// masking), then, if TAIL, one iteration in which only the first
// NQ - KF * TEAM lanes hold a quad.  d[KF] holds the tail quad.
// SIG (uncertainty weights, Eq. 12): the rows hold ore margins, the value
// term takes the weighted discount difference of the scenario from the
// period-pair row dwt[t1][t2] instead of the scalar dd, and a shift adds the
// mining-cost change cm (a swap of equal masses has none).
template <int TEAM, int KF, bool TAIL, bool SWAP, bool KAHAN, bool SIG = false>
__device__ __forceinline__ void team_eval_fast(const EvalArgs &A, int tl, const float *row1,
                                               const float *row2, uint32_t t1, uint32_t t2, float dd, float cm,
                                               int ntail, float invS, float (&d)[KF + 1][4], float &mu,
                                               float &sd) {
    const int S_pad = A.S_pad, ore_off = A.ore_off;
    const uint32_t T1 = (uint32_t)A.T + 1u;
    const float4 *r1 = reinterpret_cast<const float4 *>(row1) + tl;
    const float4 *r2 = reinterpret_cast<const float4 *>(row2) + tl;
    const uint32_t *w1 = reinterpret_cast<const uint32_t *>(row1 + ore_off);
    const uint32_t *w2 = reinterpret_cast<const uint32_t *>(row2 + ore_off);
    // period-pair rows: p12 = Pout[t1] + Pin[t2] (ore leaving t1 for t2), p21 the reverse
    const float4 *p12 = reinterpret_cast<const float4 *>(A.ctab + ((size_t)t1 * T1 + t2) * S_pad) + tl;
    const float4 *p21 = reinterpret_cast<const float4 *>(A.ctab + ((size_t)t2 * T1 + t1) * S_pad) + tl;
    const float4 *dw12 = SIG ? reinterpret_cast<const float4 *>(A.dwt + ((size_t)t1 * T1 + t2) * S_pad) + tl : nullptr;
    float sum = 0.0f, csum = 0.0f;
    const uint64_t dd2 = f2_pack(dd, dd), cm2 = f2_pack(cm, cm);
    // Where a lane's ore words are the first four of the row at known
    // positions (4-lane teams: word k / 2 in iteration k; 8-lane teams: word k,
    // at most four iterations), one 16-byte load per row fetches them all (the
    // row stride leaves four words after ore_off whenever W <= 4).
    constexpr bool ORE4 = TEAM == 4 || (TEAM == 8 && KF + (TAIL ? 1 : 0) <= 4);
    uint4 ow1 = make_uint4(0u, 0u, 0u, 0u), ow2 = ow1;
    if (ORE4) {
        ow1 = __ldg(reinterpret_cast<const uint4 *>(w1));
        if (SWAP) ow2 = __ldg(reinterpret_cast<const uint4 *>(w2));
    }
    auto word = [&](const uint4 &o, const uint32_t *w, int k, int wi) -> uint32_t {
        if (!ORE4) return __ldg(w + wi);
        const int c = TEAM == 4 ? (k >> 1) : k;
        return c == 0 ? o.x : (c == 1 ? o.y : (c == 2 ? o.z : o.w));
    };
    auto quad = [&](int k, float (&x)[4]) {
        const int q = tl + k * TEAM;
        const int wi = q >> 3;
        const uint32_t sh = (uint32_t)(q & 7) * 4u;
        const float4 a = __ldg(r1 + k * TEAM);
        const float4 pa = __ldg(p12 + k * TEAM);
        float4 w = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (SIG) w = __ldg(dw12 + k * TEAM);
        const uint64_t dlo = SIG ? f2_pack(w.x, w.y) : dd2, dhi = SIG ? f2_pack(w.z, w.w) : dd2;
        if (SWAP) {
            const float4 b = __ldg(r2 + k * TEAM);
            const uint32_t n1 = (word(ow1, w1, k, wi) >> sh) & 0xfu;
            const uint32_t n2 = (word(ow2, w2, k, wi) >> sh) & 0xfu;
            const float4 m1 = nib_mask(n1 & ~n2);
            const float4 m2 = nib_mask(n2 & ~n1);
            const float4 pb = __ldg(p21 + k * TEAM);
            // x = (a - b) dd + (m2 pb + m1 pa), scenario by scenario, in pairs
            const uint64_t lo = f2_fma(f2_sub(f2_pack(a.x, a.y), f2_pack(b.x, b.y)), dlo,
                                       f2_fma(f2_pack(m2.x, m2.y), f2_pack(pb.x, pb.y),
                                              f2_mul(f2_pack(m1.x, m1.y), f2_pack(pa.x, pa.y))));
            const uint64_t hi = f2_fma(f2_sub(f2_pack(a.z, a.w), f2_pack(b.z, b.w)), dhi,
                                       f2_fma(f2_pack(m2.z, m2.w), f2_pack(pb.z, pb.w),
                                              f2_mul(f2_pack(m1.z, m1.w), f2_pack(pa.z, pa.w))));
            f2_unpack(lo, x[0], x[1]);
            f2_unpack(hi, x[2], x[3]);
        } else {
            const float4 m1 = nib_mask((word(ow1, w1, k, wi) >> sh) & 0xfu);
            // x = a dd + m1 pa  (SIG: a dw + (m1 pa + cm))
            const uint64_t plo = SIG ? f2_fma(f2_pack(m1.x, m1.y), f2_pack(pa.x, pa.y), cm2)
                                     : f2_mul(f2_pack(m1.x, m1.y), f2_pack(pa.x, pa.y));
            const uint64_t phi = SIG ? f2_fma(f2_pack(m1.z, m1.w), f2_pack(pa.z, pa.w), cm2)
                                     : f2_mul(f2_pack(m1.z, m1.w), f2_pack(pa.z, pa.w));
            const uint64_t lo = f2_fma(f2_pack(a.x, a.y), dlo, plo);
            const uint64_t hi = f2_fma(f2_pack(a.z, a.w), dhi, phi);
            f2_unpack(lo, x[0], x[1]);
            f2_unpack(hi, x[2], x[3]);
        }
    };
    auto acc = [&](const float (&x)[4]) {
        // (x0 + x2) + (x1 + x3), the first level as one paired add; the
        // compensated form then adds the quad's sum with Kahan's update
        float u, v;
        f2_unpack(f2_add(f2_pack(x[0], x[1]), f2_pack(x[2], x[3])), u, v);
        if (KAHAN) kahan_add(sum, csum, u + v);
        else sum += u + v;
    };
#pragma unroll
    for (int k = 0; k < KF; k++) {
        quad(k, d[k]);
        acc(d[k]);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) d[KF][j] = 0.0f;
    if (TAIL && tl < ntail) {
        quad(KF, d[KF]);
        acc(d[KF]);
    }
    if (KAHAN) {
        // (sum, -csum) is a value and its error term: the team's are merged by
        // error-free TwoSum
        csum = -csum;
        team_sum_comp<TEAM>(sum, csum);
        mu = (sum + csum) * invS;
    } else {
        mu = team_sum<TEAM>(sum) * invS;
    }
    // second pass: squared deviations (non-negative terms: nothing cancels)
    float var = 0.0f;
    const uint64_t mu2 = f2_pack(mu, mu);
    auto vacc = [&](const float (&x)[4]) {
        float dv[4];
        f2_unpack(f2_sub(f2_pack(x[0], x[1]), mu2), dv[0], dv[1]);
        f2_unpack(f2_sub(f2_pack(x[2], x[3]), mu2), dv[2], dv[3]);
#pragma unroll
        for (int j = 0; j < 4; j++) var = fmaf(dv[j], dv[j], var);
    };
#pragma unroll
    for (int k = 0; k < KF; k++) vacc(d[k]);
    if (TAIL && tl < ntail) vacc(d[KF]);
    var = team_sum<TEAM>(var);
    if (KAHAN) {
        // corrected two-pass variance: minus (sum of deviations)^2 / S, the
        // bias the rounded mean leaves in the sum of squares; the deviations'
        // sum is the compensated total minus S mu (one rounding, by FMA)
        const float ds = fmaf(-(float)A.S, mu, sum) + csum;
        var = fmaxf(var - ds * ds * invS, 0.0f);
    }
    sd = sqrtf(var * invS);
}

template <int TEAM, int KF>
__device__ __forceinline__ void write_deltas_fast(const EvalArgs &A, int64_t i, int tl, int ntail,
                                                  const float (&d)[KF + 1][4]) {
    float4 *drow = reinterpret_cast<float4 *>(A.delta + i * (int64_t)A.S);
#pragma unroll
    for (int k = 0; k < KF; k++) drow[tl + k * TEAM] = make_float4(d[k][0], d[k][1], d[k][2], d[k][3]);
    if (tl < ntail) drow[tl + KF * TEAM] = make_float4(d[KF][0], d[KF][1], d[KF][2], d[KF][3]);
}

// Per-scenario deltas of one move to delta[i][0..S).
template <int TEAM, int QMAX>
__device__ __forceinline__ void write_deltas(const EvalArgs &A, int64_t i, int tl, int NQ, int rem,
                                             const float (&d)[QMAX][4]) {
    float *drow = A.delta + i * (int64_t)A.S;
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

// Non-binding prefetch of one 128-byte line into L1.
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// The lanes of a team prefetch the 128-byte lines of one block row.
template <int TEAM>
__device__ __forceinline__ void prefetch_row(const float *row, uint32_t row_bytes, int tl) {
    const uintptr_t beg = reinterpret_cast<uintptr_t>(row) & ~(uintptr_t)127;
    const uintptr_t end = reinterpret_cast<uintptr_t>(row) + row_bytes;
    for (uintptr_t a = beg + (uintptr_t)tl * 128; a < end; a += (uintptr_t)TEAM * 128)
        prefetch_l1(reinterpret_cast<const void *>(a));
}

// End of the evaluation part of a fused search step: warp 0 merges the
// warps' lists (skipping lists that cannot contribute) and writes the CTA's 32
// best keys to out32[0..32).  Every key of the batch's top k is among the 32
// best of the CTA that evaluated it; the finisher selects from these lists.
__device__ __forceinline__ void step_publish(uint64_t *out32, uint64_t wtk) {
    constexpr int NW = kEvalThreads / 32;
    __shared__ uint64_t s_wtk[NW][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s_wtk[warp][lane] = wtk;
    __syncthreads();
    if (warp == 0) {
        uint64_t t = s_wtk[0][lane];
        for (int w = 1; w < NW; w++) t = warp_topk_merge(t, s_wtk[w][lane]);
        out32[lane] = t;
    }
}

// Merge tree over the NW warps' lists (any NW >= 1): t is the calling warp's
// list, also stored in s_wl[warp]; at each level the upper half of the
// remaining lists is merged into the lower half.  With INFO the move record of
// each list's head follows it in s_inf.  Every thread must call it; the result
// is valid in warp 0 (and s_inf[0]).
template <int NW, bool INFO>
__device__ __forceinline__ uint64_t tree_merge(uint64_t t, uint64_t (*s_wl)[32], int4 *s_inf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int width = NW; width > 1; width = (width + 1) / 2) {
        const int half = (width + 1) / 2;
        if (warp < width - half) {
            const uint64_t o = s_wl[warp + half][lane];
            const uint64_t mrg = warp_topk_merge(t, o);
            if (INFO && __shfl_sync(0xffffffffu, mrg == o, 0) && lane == 0) s_inf[warp] = s_inf[warp + half];
            t = mrg;
            s_wl[warp][lane] = t;
        }
        __syncthreads();
    }
    return t;
}

// Selection of the 32 largest keys among nlists published lists (each sorted
// best-first, 0 = empty; keys unique) by the whole CTA (NW warps): warp w
// merges lists w, w + NW, ... with pruned warp merges, four lists' loads in
// flight at a time, then a tree over the warps.  Every thread
// must call it; the result is valid in warp 0 (sorted, lane 0 best).
template <int NW>
__device__ __forceinline__ uint64_t block_merge_lists(const uint64_t *lists, int nlists, uint64_t (*s_wl)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t t = 0;
    for (int l0 = warp; l0 < nlists; l0 += 4 * NW) {
        uint64_t c[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int l = l0 + u * NW;
            c[u] = l < nlists ? __ldcg(lists + (size_t)l * 32 + lane) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) t = warp_topk_merge(t, c[u]);
    }
    s_wl[warp][lane] = t;
    __syncthreads();
    return tree_merge<NW, false>(t, s_wl, nullptr);
}

// block_merge_lists that also follows the move record of the best key:
// infos[l] belongs to lists[l]'s head; the record of the merged head comes
// back in inf_out (valid in every thread after the call).
template <int NW>
__device__ __forceinline__ uint64_t block_merge_lists_info(const uint64_t *lists, const int4 *infos, int nlists,
                                                           uint64_t (*s_wl)[32], int4 *s_inf, int4 &inf_out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t t = 0;
    int4 inf = make_int4(0, 0, 0, 0);
    for (int l0 = warp; l0 < nlists; l0 += 4 * NW) {
        uint64_t c[4];
        int4 ci[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int l = l0 + u * NW;
            c[u] = l < nlists ? __ldcg(lists + (size_t)l * 32 + lane) : 0ull;
            ci[u] = l < nlists ? __ldcg(infos + l) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint64_t mrg = warp_topk_merge(t, c[u]);
            if (__shfl_sync(0xffffffffu, mrg == c[u], 0)) inf = ci[u];  // the head came from list u
            t = mrg;
        }
    }
    s_wl[warp][lane] = t;
    if (lane == 0) s_inf[warp] = inf;
    __syncthreads();
    t = tree_merge<NW, true>(t, s_wl, s_inf);
    inf_out = s_inf[0];
    return t;
}

// Called by one full warp with the merged list t: writes the top k (move
// indices, their scores decoded from the keys, the count) and returns the
// best move's index in every lane, -1 when nothing is feasible.  A key always
// decodes to a move of the batch; the range check (< n) makes sure a corrupted
// list can never turn into an out-of-range access (it raises the bad-move bit).
__device__ __forceinline__ int warp_write_topk(uint64_t t, int k, int64_t n, uint32_t *status, int32_t *idx_out,
                                               float *top_out, int32_t *count_out) {
    const int lane = threadIdx.x & 31;
    const uint32_t valid = __ballot_sync(0xffffffffu, t != 0ull);
    int cnt = min(__popc(valid), k);
    const uint32_t id = ~(uint32_t)(t & 0xffffffffull);
    const bool ok = (uint64_t)id < (uint64_t)n;
    const uint32_t bad = __ballot_sync(0xffffffffu, lane < cnt && !ok);
    if (bad) {
        cnt = __ffs(bad) - 1;
        if (lane == 0) atomicOr(status, kStBadMove);
    }
    const uint32_t id0 = __shfl_sync(0xffffffffu, id, 0);
    if (lane < cnt) {
        idx_out[lane] = (int32_t)id;
        // the key's upper half is the score's order-preserving image: invert
        // it (a -0.0 score, folded into +0.0 by the key, comes back as +0.0)
        const uint32_t ord = (uint32_t)(t >> 32);
        top_out[lane] = __uint_as_float((ord & 0x80000000u) ? (ord & 0x7fffffffu) : ~ord);
    }
    if (lane == 0) *count_out = cnt;
    return cnt > 0 ? (int)id0 : -1;
}

// Ticket counter increment with acquire-release semantics at GPU scope: it
// publishes what the calling CTA wrote before its barrier (release is
// cumulative over the barrier) and makes visible what the CTAs that drew the
// earlier numbers published.
__device__ __forceinline__ uint32_t ticket_next(uint32_t *p) {
    uint32_t old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

// Non-binding prefetch into L2 of [p, p + bytes), 128-byte lines; thread i of
// nt takes lines i, i + nt, ...
__device__ __forceinline__ void prefetch_l2_range(const void *p, size_t bytes, int i, int nt) {
    const char *c = static_cast<const char *>(p);
    for (size_t o = (size_t)i * 128; o < bytes; o += (size_t)nt * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// End of a standalone top-k selection (k_topk_lists), called by every thread
// of every CTA with the warp's list wtk.  The CTA merges its warps' lists (a
// tree) and publishes its 32 best keys; the last CTA of each group of
// grp_size CTAs to finish (a ticket counter per group; nobody waits) merges
// the group's lists into one; the last group to finish merges the group lists
// and writes the top k.  Each ticket is reset by the CTA that draws its last
// number, so every counter is zero again for the next launch.  Two levels of
// about sqrt(grid) lists each keep the merging short, and all but the last
// group merge while others still run.  Not inlined: the caller's main loop
// keeps its own register allocation.
static __device__ __noinline__ void step_reduce(const StepTail &T, uint64_t wtk) {
    constexpr int NW = kEvalThreads / 32;
    __shared__ uint64_t s_wl[NW][32];
    __shared__ int s_last;
    const StepLists &L = T.L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_wl[warp][lane] = wtk;
    __syncthreads();
    wtk = tree_merge<NW, false>(wtk, s_wl, nullptr);
    if (warp == 0) L.cta[(size_t)blockIdx.x * 32 + lane] = wtk;
    __syncthreads();
    const int g = (int)blockIdx.x / L.grp_size, g0 = g * L.grp_size;
    const int gn = min(L.grp_size, (int)gridDim.x - g0);
    const int ng = ((int)gridDim.x + L.grp_size - 1) / L.grp_size;
    if (tid == 0) s_last = ticket_next(L.tick + g) == (uint32_t)(gn - 1);
    __syncthreads();
    if (!s_last) return;
    uint64_t t = block_merge_lists<NW>(L.cta + (size_t)g0 * 32, gn, s_wl);
    if (warp == 0) L.grp[(size_t)g * 32 + lane] = t;
    if (tid == 0) L.tick[g] = 0;
    __syncthreads();
    if (tid == 0) s_last = ticket_next(L.tick + L.final_slot) == (uint32_t)(ng - 1);
    __syncthreads();
    if (!s_last) return;
    t = block_merge_lists<NW>(L.grp, ng, s_wl);
    if (warp == 0) warp_write_topk(t, T.k, T.n, T.status, T.idx_out, T.top_out, T.count_out);
    if (tid == 0) L.tick[L.final_slot] = 0;
}

// Per-warp lists and staging of the evaluator (static shared memory).
template <int NW>
struct EvalSharedT {
    int32_t b1[NW][kChunk], b2[NW][kChunk];
    uint32_t tt[NW][kChunk];
    uint8_t lsh[NW][kChunk], lsw[NW][kChunk];
    float score[NW][kChunk], mean[NW][kChunk];
    uint8_t flag[NW][kChunk];
    int4 best[NW];  // TOPK: the move of the warp's best key (b1, b2 or B, t1 | t2 << 8, 0)
};
using EvalShared = EvalSharedT<kEvalThreads / 32>;

// Static shared memory of an evaluator CTA.  The fused step's final CTA reuses
// the per-warp staging once every warp has finished evaluating, for the
// batch's selection and the apply.
template <int NW>
struct EvalSmemPlain {
    EvalSharedT<NW> ev;
};
template <int NW>
union EvalSmemStep {
    EvalSharedT<NW> ev;
    float apply_tab[kApplyTabMax];
};

// End of the fused search step, called by every thread of every CTA (NW warps,
// one CTA per SM) with the warp's list wtk and the move record of each warp's
// best key (winfo[warp], shared memory).  su: the CTA's shared staging, free
// for reuse once every warp has arrived here (the final CTA's selection and
// apply use it).
//   0. The first warp of the CTA to finish evaluating (s_fin, a shared counter
//      zeroed at the CTA's start) does the CTA's share of the FP64 update the
//      previous step left due (*pending): metal, net cash and NPV_s of
//      scenarios blockIdx.x, blockIdx.x + gridDim.x, ..., while the CTA's
//      other warps still evaluate.
//   1. The CTA merges its warps' lists (a tree of warp merges, keeping the
//      record of the best key), publishes the result and that record,
//      prefetches its share of the state the final apply touches into L2, and
//      draws the final ticket (acquire-release; nobody waits).
//   2. The CTA that draws the last number ranks the lists' heads (only lists
//      whose heads rank among the 32 best can hold one of the 32 best keys),
//      selects the 32 best keys of those lists (the keys no smaller than the
//      32nd head, each ranked against the others; a tree of warp merges when
//      there are many), writes the top k, applies
//      the structural part of the best move from its record (tonnage, schedule
//      words, penalty tables: all the next evaluation reads) and leaves the
//      move's FP64 part due in *pending (or clears *pending without an apply).
// Counters are reset by the final CTA.  Not inlined: the evaluator's main loop
// keeps its own register allocation.
template <int NW>
static __device__ __noinline__ void step_finish(const StepTail &T, uint64_t wtk, const int4 *winfo,
                                                EvalSmemStep<NW> &su, uint32_t *s_fin) {
    constexpr int NT = NW * 32;
    __shared__ uint64_t s_wl[NW][32];
    __shared__ int4 s_inf[NW];
    __shared__ uint64_t s_heads[256];  // grids of up to 256 CTAs (one per SM)
    __shared__ int s_slot[32];
    __shared__ int4 s_best_inf;
    __shared__ int s_last, s_best, s_ncand;
    const StepLists &L = T.L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t order = 0u;
    if (lane == 0) order = atomicAdd(s_fin, 1u);
    if (__shfl_sync(0xffffffffu, order, 0) == 0u) {
        const int4 pend = *T.pending;
        if (pend.w) apply_money(T.ap, pend, (int)blockIdx.x + lane * (int)gridDim.x, 32 * (int)gridDim.x);
    }
    s_wl[warp][lane] = wtk;
    if (lane == 0) s_inf[warp] = winfo[warp];
    __syncthreads();
    // 1. the CTA's 32 best keys: a tree of warp merges
    wtk = tree_merge<NW, true>(wtk, s_wl, s_inf);
    if (warp == 0) {
        L.cta[(size_t)blockIdx.x * 32 + lane] = wtk;
        if (lane == 0) L.cinf[blockIdx.x] = s_inf[0];  // unused when the list is empty
    }
    if (T.do_apply) {
        const ApplyArgs &P = T.ap;
        const int i = (int)blockIdx.x * NT + tid, nt = (int)gridDim.x * NT;
        prefetch_l2_range(P.oreT, (size_t)(P.T + 1) * P.S * sizeof(int64_t), i, nt);
        prefetch_l2_range(P.tab, (size_t)2 * (P.T + 1) * P.S_pad * sizeof(float), i, nt);
        prefetch_l2_range(P.blk, (size_t)P.tp.B * sizeof(uint32_t), i, nt);
    }
    __syncthreads();
    if (tid == 0) s_last = ticket_next(L.tick + L.final_slot) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    // 2. the batch's top k
    const int G = (int)gridDim.x;
    int4 inf;
    uint64_t t;
    if (G <= 256) {
        // Only a list whose head is among the 32 best heads can hold one of
        // the 32 best keys (those heads are 32 keys at least as large as any
        // key of a list below them): rank the heads, then merge those lists.
        uint64_t head = 0ull;
        int4 my_inf = make_int4(0, 0, 0, 0);
        if (tid < G) {
            head = __ldcg(L.cta + (size_t)tid * 32);
            my_inf = __ldcg(L.cinf + tid);
            s_heads[tid] = head;
        }
        const int nonempty = __syncthreads_count(head != 0ull);
        if (tid < G && head != 0ull) {
            int r = 0;
            for (int j = 0; j < G; j++) r += s_heads[j] > head ? 1 : 0;
            if (r < 32) {
                s_slot[r] = tid;
                if (r == 0) s_best_inf = my_inf;  // the best key heads its CTA's list
            }
        }
        if (tid == 0) s_ncand = 0;
        __syncthreads();
        const int nc = min(nonempty, 32);
        // With 32 lists selected, their 32 heads are keys at least as large as
        // the smallest of them (tau), so the 32 best keys are all >= tau: they
        // are found among the keys >= tau of the selected lists (few, unless
        // many keys lie close together), each ranked by comparison with the
        // others.  With fewer lists every key is a candidate.  Too many
        // candidates for the staging (s_wl, free again here) fall back to a
        // merge tree; both give the same sorted 32 keys (keys are unique).
        const uint64_t tau = nc == 32 ? s_heads[s_slot[31]] : 1ull;
        uint64_t *s_cand = &s_wl[0][0];
        constexpr int kCandMax = NW * 32 < 256 ? NW * 32 : 256;
        for (int r = warp; r < nc; r += NW) {
            const uint64_t key = __ldcg(L.cta + (size_t)s_slot[r] * 32 + lane);
            const uint32_t m = __ballot_sync(0xffffffffu, key >= tau);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&s_ncand, __popc(m));
            const int pos = __shfl_sync(0xffffffffu, base, 0) + __popc(m & ((1u << lane) - 1u));
            if (key >= tau && pos < kCandMax) s_cand[pos] = key;
        }
        __syncthreads();
        const int ncand = s_ncand;
        __syncthreads();  // every thread has read the count before the tree may reuse s_wl
        if (ncand <= kCandMax) {
            uint64_t *s_out = s_heads;  // the heads are no longer read
            if (tid < ncand) {
                const uint64_t key = s_cand[tid];
                int r = 0;
                for (int j = 0; j < ncand; j++) r += s_cand[j] > key ? 1 : 0;
                if (r < 32) s_out[r] = key;
            }
            if (tid >= ncand && tid < 32) s_out[tid] = 0ull;
            __syncthreads();
            t = warp == 0 ? s_out[lane] : 0ull;
        } else {
            // warp w < 16 merges the lists of ranks 2w and 2w + 1, then a tree
            t = 0ull;
            if (warp < 16) {
                const uint64_t a = 2 * warp < nc ? __ldcg(L.cta + (size_t)s_slot[2 * warp] * 32 + lane) : 0ull;
                const uint64_t b = 2 * warp + 1 < nc ? __ldcg(L.cta + (size_t)s_slot[2 * warp + 1] * 32 + lane) : 0ull;
                t = warp_topk_merge(a, b);
                s_wl[warp][lane] = t;
            }
            __syncthreads();
            t = tree_merge<(NW < 16 ? NW : 16), false>(t, s_wl, nullptr);
        }
        inf = s_best_inf;
    } else {
        t = block_merge_lists_info<NW>(L.cta, L.cinf, G, s_wl, s_inf, inf);
    }
    if (warp == 0) {
        const int best = warp_write_topk(t, T.k, T.n, T.status, T.idx_out, T.top_out, T.count_out);
        if (lane == 0) s_best = best;
    }
    if (tid == 0) L.tick[L.final_slot] = 0;
    if (!T.do_apply) {
        if (tid == 0) T.pending->w = 0;  // every CTA has read it
        return;
    }
    __syncthreads();
    const int changed = apply_evaluated<false>(T.ap, inf, s_best >= 0 ? 1 : 0, su.apply_tab);
    if (tid == 0) *T.pending = make_int4(inf.x, inf.y, inf.z, changed);
}

// List storage and tickets of model m for a launch of `grid` CTAs (mm_eval.cu).
StepLists step_lists(mm_model *m, int grid);

// Move i of the batch, from the 8-byte or the compact 4-byte form.
__device__ __forceinline__ int2 load_move(const EvalArgs &A, int64_t i) {
    return A.pmoves ? unpack_move(__ldg(A.pmoves + i), A.tp.B, A.tp.T) : __ldg(A.moves + i);
}

// Evaluator arguments for a batch of n moves on model m (mm_eval.cu).
EvalArgs eval_args(mm_model *m, const mm_move *moves, int64_t n, float *score, uint8_t *feas, float *mean,
                   float *delta);


// The evaluator proper: the calling warp evaluates moves [r0, r1) of A in
// chunks of 64 (decode two per lane, shift / swap lists by ballot, teams of
// TEAM lanes per move, coalesced stores) and, if TOPK, inserts every feasible
// move's key into its register list wtk.  tab, s_dd, s_mined and s_cap are
// the CTA's staged tables.
template <int TEAM, int QMAX, bool KAHAN, bool DELTA, int KF, bool TAIL, bool TOPK, bool SIG = false,
          int NW = kEvalThreads / 32>
__device__ __forceinline__ void eval_warp_range(const EvalArgs &A, EvalSharedT<NW> &sh, const float *tab, const float *s_dd,
                                                const int64_t *s_mined, const uint64_t *s_cap, int64_t r0, int64_t r1,
                                                uint64_t &wtk, const int2 *first = nullptr) {
    constexpr int CH = kChunk;
    constexpr int TPW = 32 / TEAM;
    const int T1 = A.T + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tl = lane % TEAM, tw = lane / TEAM;
    const int S = A.S;
    const int NQ = (S + 3) >> 2;
    const int rem = S - 4 * (NQ - 1);
    const float invS = 1.0f / (float)S;
    const size_t pin_off = (size_t)T1 * A.S_pad;
    const uint32_t lt_mask = (1u << lane) - 1u;
    // the first chunk's moves (first: loaded by the caller before its set-up)
    int2 mv[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int64_t i = r0 + h * 32 + lane;
        mv[h] = first ? first[h] : (i < r1 ? load_move(A, i) : make_int2(0, -1));
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
            mv[h] = ni < r1 ? load_move(A, ni) : make_int2(0, -1);
            const bool work = active && v.valid && !v.noop;
            if (active) {
                A.feas[i] = v.feasible ? 1 : 0;
                if (!v.valid) atomicOr(A.status, kStBadMove);
                if (DELTA && !work) {
                    float *drow = A.delta + i * (int64_t)S;
                    for (int s2 = 0; s2 < S; s2++) drow[s2] = 0.0f;
                }
            }
            sh.score[warp][slot] = v.valid ? 0.0f : -INFINITY;
            sh.mean[warp][slot] = 0.0f;
            if (TOPK) sh.flag[warp][slot] = (active && v.feasible) ? 1 : 0;
            if (active && v.valid) {  // every feasible move's data, for the top-k's move record
                sh.b1[warp][slot] = v.b1;
                sh.b2[warp][slot] = v.swap ? v.b2 : A.tp.B;
                sh.tt[warp][slot] = v.t1 | (v.t2 << 8);
            }
            const bool is_sh = work && !v.swap, is_sw = work && v.swap;
            const uint32_t msh = __ballot_sync(0xffffffffu, is_sh);
            const uint32_t msw = __ballot_sync(0xffffffffu, is_sw);
            if (is_sh) sh.lsh[warp][nsh + __popc(msh & lt_mask)] = (uint8_t)slot;
            if (is_sw) sh.lsw[warp][nsw + __popc(msw & lt_mask)] = (uint8_t)slot;
            nsh += __popc(msh);
            nsw += __popc(msw);
        }
        __syncwarp();
        // ---- compute: batches of TPW list entries, shifts first, then swaps;
        //      the rows of batch j + prefetch are pulled into L1 meanwhile ----
        const int nbs = (nsh + TPW - 1) / TPW, nb = nbs + (nsw + TPW - 1) / TPW;
        const uint32_t row_bytes = (uint32_t)A.R * 4u;
        auto prefetch_batch = [&](int j) {
            if (j >= nb) return;
            const bool sw = j >= nbs;
            const int e = (sw ? j - nbs : j) * TPW + tw;
            if (e < (sw ? nsw : nsh)) {
                const int slot = (sw ? sh.lsw[warp] : sh.lsh[warp])[e];
                prefetch_row<TEAM>(A.val + (size_t)sh.b1[warp][slot] * A.R, row_bytes, tl);
                if (sw) prefetch_row<TEAM>(A.val + (size_t)sh.b2[warp][slot] * A.R, row_bytes, tl);
            }
        };
        for (int j = 0; j < A.prefetch && j < nb; j++) prefetch_batch(j);
#pragma unroll 1
        for (int j = 0; j < nb; j++) {
            if (A.prefetch > 0) prefetch_batch(j + A.prefetch);
            const bool sw = j >= nbs;
            const int e = (sw ? j - nbs : j) * TPW + tw;
            const int nl = sw ? nsw : nsh;
            const bool act = e < nl;
            const int slot = act ? (sw ? sh.lsw[warp] : sh.lsh[warp])[e] : 0;
            const int32_t b1 = act ? sh.b1[warp][slot] : 0;
            const int32_t b2 = act ? sh.b2[warp][slot] : 0;
            const uint32_t tt = act ? sh.tt[warp][slot] : 0;
            const uint32_t t1 = tt & 0xffu, t2 = tt >> 8;
            const float dd = s_dd[t1 * T1 + t2];
            float mu, sd;
            const float *row1 = A.val + (size_t)b1 * A.R;
            const float *row2 = A.val + (size_t)b2 * A.R;
            if constexpr (KF > 0) {
                // fast form: S % 4 == 0, KF full quad iterations, optional tail
                const int ntail = NQ - KF * TEAM;
                float d[KF + 1][4];
                if (!sw)
                    team_eval_fast<TEAM, KF, TAIL, false, KAHAN, SIG>(A, tl, row1, row2, t1, t2, dd,
                                                                      SIG ? -A.mcm * dd : 0.0f, ntail, invS, d, mu,
                                                                      sd);
                else
                    team_eval_fast<TEAM, KF, TAIL, true, KAHAN, SIG>(A, tl, row1, row2, t1, t2, dd, 0.0f, ntail,
                                                                     invS, d, mu, sd);
                if (act && DELTA) write_deltas_fast<TEAM, KF>(A, c0 + slot, tl, ntail, d);
            } else {
                static_assert(!SIG, "the weighted form is the fast form only");
                float d[QMAX][4];
                if (!sw)
                    team_eval<TEAM, QMAX, false, KAHAN, false>(A, tab, tl, act, row1, row2, t1, t2, dd, NQ,
                                                               rem, invS, pin_off, d, mu, sd);
                else
                    team_eval<TEAM, QMAX, true, KAHAN, false>(A, tab, tl, act, row1, row2, t1, t2, dd, NQ,
                                                              rem, invS, pin_off, d, mu, sd);
                if (act && DELTA) write_deltas<TEAM, QMAX>(A, c0 + slot, tl, NQ, rem, d);
            }
            if (act && tl == 0) {
                sh.score[warp][slot] = mu - A.lambda * sd;
                sh.mean[warp][slot] = mu;
            }
        }
        __syncwarp();
        // ---- store (coalesced) ----
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int slot = h * 32 + lane;
            const int64_t i = c0 + slot;
            if (i < r1) {
                A.score[i] = sh.score[warp][slot];
                if (A.mean) A.mean[i] = sh.mean[warp][slot];
            }
            if (TOPK) {
                uint64_t key = 0;
                if (i < r1 && sh.flag[warp][slot]) {
                    const float f = sh.score[warp][slot];
                    if (!isnan(f)) key = score_key(f, i);
                }
                const uint64_t before = __shfl_sync(0xffffffffu, wtk, 0);
                wtk = warp_topk_insert(wtk, key);
                const uint64_t after = __shfl_sync(0xffffffffu, wtk, 0);
                if (after != before) {
                    // a new best came from this round: record its move
                    const int src = __ffs(__ballot_sync(0xffffffffu, key == after)) - 1;
                    const int sl = h * 32 + src;
                    if (lane == 0) sh.best[warp] = make_int4(sh.b1[warp][sl], sh.b2[warp][sl], (int)sh.tt[warp][sl], 0);
                }
            }
        }
        __syncwarp();
    }
}

template <int TEAM, int QMAX, bool KAHAN, bool DELTA, bool TSM, int KF = 0, bool TAIL = false, bool TOPK = false,
          bool SIG = false, int NT = kEvalThreads>
__global__ void __launch_bounds__(NT, NT == kEvalThreads ? MM_EVAL_MINB : 1) k_eval_tiled(EvalArgs A) {
    constexpr int NW = NT / 32;   // warps per CTA
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) std::conditional_t<TOPK, EvalSmemStep<NW>, EvalSmemPlain<NW>> su;
    EvalSharedT<NW> &sh = su.ev;

    const int T1 = A.T + 1;
    const size_t tab_floats = (size_t)2 * T1 * A.S_pad;
    float *s_tab = reinterpret_cast<float *>(smem);                            // [2][T+1][S_pad] if TSM
    float *s_dd = s_tab + (TSM ? tab_floats : 0);                              // [(T+1)^2] if dd_smem
    size_t off = ((TSM ? tab_floats : 0) + (A.dd_smem ? (size_t)T1 * T1 : 0)) * sizeof(float);
    off = (off + 15) & ~(size_t)15;
    int64_t *s_mined = reinterpret_cast<int64_t *>(smem + off);                // [T+1]
    uint64_t *s_cap = reinterpret_cast<uint64_t *>(s_mined + T1);              // [T+1]

    const int tid = threadIdx.x;
    // contiguous, balanced range of moves for each warp; its first moves'
    // loads go out before the set-up below, so their latency overlaps it
    const int warp = tid >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * NW;
    const int64_t gw = (int64_t)blockIdx.x * NW + warp;
    const int64_t r0 = gw * A.n / nwarps, r1 = (gw + 1) * A.n / nwarps;
    int2 first[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int64_t i = r0 + h * 32 + (tid & 31);
        first[h] = i < r1 ? load_move(A, i) : make_int2(0, -1);
    }
    __shared__ uint32_t s_fin;  // TOPK: warps of this CTA that have finished evaluating
    if (TOPK && tid == 0) s_fin = 0u;
    if (TSM) {
        const float4 *src = reinterpret_cast<const float4 *>(A.tab);
        float4 *dst = reinterpret_cast<float4 *>(s_tab);
        for (int i = tid; i < (int)(tab_floats / 4); i += NT) dst[i] = __ldg(src + i);
    }
    if (A.dd_smem)
        for (int i = tid; i < T1 * T1; i += NT) s_dd[i] = __ldg(A.ddt + i);
    for (int i = tid; i < T1; i += NT) {
        s_mined[i] = A.minedT[i];
        s_cap[i] = A.cap[i];
    }
    __syncthreads();
    const float *tab = TSM ? s_tab : A.tab;
    uint64_t wtk = 0;  // this warp's best 32 candidate keys (TOPK)
    eval_warp_range<TEAM, QMAX, KAHAN, DELTA, KF, TAIL, TOPK, SIG, NW>(A, sh, tab, A.dd_smem ? s_dd : A.ddt,
                                                                       s_mined, s_cap, r0, r1, wtk, first);
    if constexpr (TOPK) step_finish<NW>(A.tail, wtk, sh.best, su, &s_fin);
}

// ----------------------------------------------------------------------------
// Bulk-copy (TMA) staged evaluator.  Same decode / list / team structure as
// k_eval_tiled, but the value rows of the next batches of moves are copied
// into shared memory by cp.async.bulk (one 1-D copy per moved block row,
// values and ore bits together), tracked by one mbarrier per pipeline stage,
// so the gathers of several batches are in flight while a batch is computed.
// A batch is TPW = 32 / TEAM list entries (one per team).  Lane 0 of the warp
// is the producer.  Every wait is bounded: on expiry the kernel raises the
// sticky timeout bit, drains its own copies (again bounded) and returns.

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before its
// later async-proxy (bulk copy) accesses to the same buffers.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: far beyond any legitimate copy latency
constexpr long long kTestWaitCycles = 2000000LL;  // ~1 ms: the test-only stall mode's limit

// Bounded wait for a pipeline stage (uniform across the warp): false when
// `limit` clock cycles pass first.
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity, long long limit) {
    bool ok = mbar_try_wait(bar, parity);
    if (!ok) {
        const long long t0 = clock64();
        while (!(ok = mbar_try_wait(bar, parity)))
            if (clock64() - t0 > limit) break;
    }
    return __all_sync(0xffffffffu, ok);
}

constexpr int kMaxStages = 4;
constexpr int kDefaultStages = 0;    // direct loads measured faster than bulk copies of 416-byte rows
// The (T+1)^2 table of discount differences is staged in shared memory while
// it takes at most this many bytes (T <= 89); above, the kernels read it from
// global memory through L1 (at T = 254 it would take 254 KB).
constexpr size_t kDdSmemMax = 32 * 1024;

// Built-in L1 prefetch distance (batches ahead): none while the value rows fit
// in L2 (there the prefetches only add L1 traffic), one batch once they exceed
// it and the gathers come from DRAM (measured: 50k blocks x 100 scenarios is
// fastest at 0; 400k blocks x 500 scenarios gains ~6 % at 1, less at 2, and
// loses from 3 on).
constexpr int kPrefetchDram = 1;

template <int TEAM, int QMAX, bool KAHAN, bool DELTA, bool TSM>
__global__ void __launch_bounds__(kEvalThreads, 1) k_eval_tma(EvalArgs A) {
    constexpr int CH = kChunk;
    constexpr int NWMAX = kEvalThreads / 32;
    constexpr int TPW = 32 / TEAM;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int32_t s_b1[NWMAX][CH], s_b2[NWMAX][CH];
    __shared__ uint32_t s_tt[NWMAX][CH];
    __shared__ uint8_t s_lsh[NWMAX][CH], s_lsw[NWMAX][CH];
    __shared__ float s_score[NWMAX][CH], s_mean[NWMAX][CH];
    __shared__ __align__(8) uint64_t s_bar[NWMAX][kMaxStages];

    const int NW = blockDim.x >> 5;
    const int NS = A.nstage;
    const int T1 = A.T + 1;
    const int R = A.R;
    const size_t tab_floats = (size_t)2 * T1 * A.S_pad;
    float *s_tab = reinterpret_cast<float *>(smem);                            // [2][T+1][S_pad] if TSM
    float *s_dd = s_tab + (TSM ? tab_floats : 0);                              // [(T+1)^2] if dd_smem
    size_t off = ((TSM ? tab_floats : 0) + (A.dd_smem ? (size_t)T1 * T1 : 0)) * sizeof(float);
    off = (off + 15) & ~(size_t)15;
    int64_t *s_mined = reinterpret_cast<int64_t *>(smem + off);                // [T+1]
    uint64_t *s_cap = reinterpret_cast<uint64_t *>(s_mined + T1);              // [T+1]
    off += 2 * (size_t)T1 * sizeof(int64_t);
    off = (off + 127) & ~(size_t)127;
    float *s_stage_all = reinterpret_cast<float *>(smem + off);                // [NW][NS][TPW][2][R]

    const int tid = threadIdx.x;
    if (TSM) {
        const float4 *src = reinterpret_cast<const float4 *>(A.tab);
        float4 *dst = reinterpret_cast<float4 *>(s_tab);
        for (int i = tid; i < (int)(tab_floats / 4); i += blockDim.x) dst[i] = __ldg(src + i);
    }
    if (A.dd_smem)
        for (int i = tid; i < T1 * T1; i += blockDim.x) s_dd[i] = __ldg(A.ddt + i);
    const float *dd_tab = A.dd_smem ? s_dd : A.ddt;
    for (int i = tid; i < T1; i += blockDim.x) {
        s_mined[i] = A.minedT[i];
        s_cap[i] = A.cap[i];
    }
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
        for (int st = 0; st < NS; st++) mbar_init(&s_bar[warp][st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    const float *tab = TSM ? s_tab : A.tab;

    const int tl = lane % TEAM, tw = lane / TEAM;
    const int S = A.S;
    const int NQ = (S + 3) >> 2;
    const int rem = S - 4 * (NQ - 1);
    const float invS = 1.0f / (float)S;
    const size_t pin_off = (size_t)T1 * A.S_pad;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t row_bytes = (uint32_t)R * 4u;
    float *stage0 = s_stage_all + (size_t)warp * NS * TPW * 2 * R;
    const int64_t nwarps = (int64_t)gridDim.x * NW;
    const int64_t gw = (int64_t)blockIdx.x * NW + warp;
    const int64_t r0 = gw * A.n / nwarps, r1 = (gw + 1) * A.n / nwarps;
    uint32_t parity = 0;  // bit st: parity of the next completion of stage st
    uint32_t cnt = 0;     // batches issued (== consumed at chunk boundaries) by this warp

    int2 mv[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int64_t i = r0 + h * 32 + lane;
        mv[h] = i < r1 ? load_move(A, i) : make_int2(0, -1);
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
            const int64_t ni = i + CH;
            mv[h] = ni < r1 ? load_move(A, ni) : make_int2(0, -1);
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
        const int nbs = (nsh + TPW - 1) / TPW, nbw = (nsw + TPW - 1) / TPW, nb = nbs + nbw;
        // producer: issue batch j of this chunk into stage (cnt0 + j) % NS
        const uint32_t cnt0 = cnt;
        auto issue = [&](int j) {
            if (lane == 0) {
                const bool sw = j >= nbs;
                const uint8_t *list = sw ? s_lsw[warp] : s_lsh[warp];
                const int e0 = (sw ? j - nbs : j) * TPW, nl = sw ? nsw : nsh;
                const int st = (int)((cnt0 + (uint32_t)j) % (uint32_t)NS);
                float *buf = stage0 + (size_t)st * TPW * 2 * R;
                int ne = nl - e0 < TPW ? nl - e0 : TPW;
                fence_proxy_async();
                mbar_arrive_expect_tx(&s_bar[warp][st], (uint32_t)ne * row_bytes * (sw ? 2u : 1u) + A.tx_extra);
                for (int t = 0; t < ne; t++) {
                    const int slot = list[e0 + t];
                    bulk_copy_g2s(buf + (size_t)t * 2 * R, A.val + (size_t)s_b1[warp][slot] * R, row_bytes,
                                  &s_bar[warp][st]);
                    if (sw)
                        bulk_copy_g2s(buf + (size_t)t * 2 * R + R, A.val + (size_t)s_b2[warp][slot] * R, row_bytes,
                                      &s_bar[warp][st]);
                }
            }
        };
        for (int j = 0; j < nb && j < NS; j++) issue(j);
        cnt += (uint32_t)nb;
        bool timed_out = false;
#pragma unroll 1
        for (int j = 0; j < nb; j++) {
            const int st = (int)((cnt0 + (uint32_t)j) % (uint32_t)NS);
            if (!stage_wait(&s_bar[warp][st], (parity >> st) & 1u, A.wait_cycles)) {
                timed_out = true;
                // drain this warp's copies in flight (bounded), then leave
                for (int jj = j; jj < nb && jj < j + NS; jj++) {
                    const int st2 = (int)((cnt0 + (uint32_t)jj) % (uint32_t)NS);
                    stage_wait(&s_bar[warp][st2], (parity >> st2) & 1u, A.wait_cycles);
                }
                break;
            }
            parity ^= 1u << st;
            const bool sw = j >= nbs;
            const uint8_t *list = sw ? s_lsw[warp] : s_lsh[warp];
            const int e = (sw ? j - nbs : j) * TPW + tw;
            const int nl = sw ? nsw : nsh;
            const bool act = e < nl;
            const int slot = act ? list[e] : 0;
            const uint32_t tt = act ? s_tt[warp][slot] : 0;
            const uint32_t t1 = tt & 0xffu, t2 = tt >> 8;
            const float dd = dd_tab[t1 * T1 + t2];
            const float *row1 = stage0 + ((size_t)st * TPW + tw) * 2 * R;
            const float *row2 = row1 + R;
            float d[QMAX][4];
            float mu, sd;
            if (!sw)
                team_eval<TEAM, QMAX, false, KAHAN, true>(A, tab, tl, act, row1, row2, t1, t2, dd, NQ, rem,
                                                          invS, pin_off, d, mu, sd);
            else
                team_eval<TEAM, QMAX, true, KAHAN, true>(A, tab, tl, act, row1, row2, t1, t2, dd, NQ, rem,
                                                         invS, pin_off, d, mu, sd);
            if (act) {
                if (tl == 0) {
                    s_score[warp][slot] = mu - A.lambda * sd;
                    s_mean[warp][slot] = mu;
                }
                if (DELTA) write_deltas<TEAM, QMAX>(A, c0 + slot, tl, NQ, rem, d);
            }
            __syncwarp();
            if (j + NS < nb) issue(j + NS);
        }
        if (timed_out) {
            if (lane == 0) atomicOr(A.status, kStTimeout);
            return;
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
