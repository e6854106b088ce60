// Device-side pieces of the schedule state shared by the model kernels, the
// apply kernel and the fused search step: ore bits of the combined rows,
// penalty arithmetic, NPV contributions and the block-level apply.
#pragma once

#include "mm_internal.cuh"
#include "mm_move.cuh"

namespace mm {

__device__ __forceinline__ uint32_t ore_bit(const float *val, int32_t R, int32_t ore_off, int32_t b, int s) {
    return (reinterpret_cast<const uint32_t *>(val + (int64_t)b * R + ore_off)[s >> 5] >> (s & 31)) & 1u;
}

// pen(x0) - pen(x1) for excess x = O - Q (exact integer parts, then FP64).
__device__ __forceinline__ double pen_diff(int64_t x0, int64_t x1, double a, double e) {
    int64_t s0 = x0 < 0 ? -x0 : 0, s1 = x1 < 0 ? -x1 : 0;
    int64_t e0 = x0 > 0 ? x0 : 0, e1 = x1 > 0 ? x1 : 0;
    return __dadd_rn(__dmul_rn(a, (double)(s0 - s1)), __dmul_rn(e, (double)(e0 - e1)));
}

__device__ __forceinline__ double pen_of(int64_t x, double a, double e) {
    return x < 0 ? __dmul_rn(a, (double)(-x)) : __dmul_rn(e, (double)x);
}

// Pout[t][s] = d_t (pen(x) - pen(x - m)), Pin[t][s] = d_t (pen(x) - pen(x + m))
// with x = oreT[t][s] - Q_t; zero for t = T and for padding scenarios.
__device__ __forceinline__ void table_entry(int t, int s, int32_t S, int32_t S_pad, int32_t T, const int64_t *oreT,
                                            const uint64_t *target, const double *disc, int64_t m, double a,
                                            double e, float *tab) {
    float po = 0.0f, pi = 0.0f;
    if (t < T && s < S) {
        int64_t x = oreT[(int64_t)t * S + s] - (int64_t)target[t];
        double d = disc[t];
        po = __double2float_rn(__dmul_rn(d, pen_diff(x, x - m, a, e)));
        pi = __double2float_rn(__dmul_rn(d, pen_diff(x, x + m, a, e)));
    }
    tab[(int64_t)t * S_pad + s] = po;
    tab[(int64_t)(T + 1) * S_pad + (int64_t)t * S_pad + s] = pi;
}

// The four x-independent table entries of period t (see table_store_c):
// Pout at x = m (any x >= m), Pout at x = 0 (any x <= 0), Pin at x = 0 (any
// x >= 0), Pin at x = -m (any x <= -m); zero for t = T.
__device__ __forceinline__ float4 table_consts(int t, int32_t T, const double *disc, int64_t m, double a, double e) {
    if (t >= T) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const double d = disc[t];
    return make_float4(__double2float_rn(__dmul_rn(d, pen_diff(m, 0, a, e))),
                       __double2float_rn(__dmul_rn(d, pen_diff(0, -m, a, e))),
                       __double2float_rn(__dmul_rn(d, pen_diff(0, m, a, e))),
                       __double2float_rn(__dmul_rn(d, pen_diff(-m, 0, a, e))));
}

// Discounted net cash of a period from its accumulators (pure form):
//   d_t (sig (price*rec*metal - pc*ore_t) - mc*mined_t - pen_t(ore_t)),
// sig = the uncertainty weight sigma(s,t) of Eq. 12 on the processing margin
// (1 without weights; 1 * x == x, so the unweighted result is unchanged).
__device__ __forceinline__ double contrib_val(int64_t o, double metal, int64_t mined, int64_t target, double disc,
                                              double pr, double pc, double mc, double a, double e, double sig) {
    double margin = __dsub_rn(__dmul_rn(pr, metal), __dmul_rn(pc, (double)o));
    double cash = __dsub_rn(__dmul_rn(sig, margin), __dmul_rn(mc, (double)mined));
    return __dmul_rn(disc, __dsub_rn(cash, pen_of(o - target, a, e)));
}

// contrib_val in FP32 throughout (the FP32 shadow accumulators).
__device__ __forceinline__ float contrib_val_f32(int64_t o, float metal, int64_t mined, int64_t target, double disc,
                                                double pr, double pc, double mc, double a, double e, double sig) {
    const float of = (float)o, dev = (float)(o - target);
    const float cash = (float)sig * ((float)pr * metal - (float)pc * of) - (float)mc * (float)mined;
    const float pen = dev < 0.0f ? (float)a * -dev : (float)e * dev;
    return (float)disc * (cash - pen);
}

// Discounted net cash of period t in scenario s (contrib_val with the state
// arrays; sig = nullptr: no uncertainty weights).
__device__ __forceinline__ double contrib_of(int t, int s, int32_t S, const double *disc, const double *metal,
                                             const int64_t *oreT, const int64_t *minedT, const uint64_t *target,
                                             double pr, double pc, double mc, double a, double e, const double *sig) {
    const int64_t i = (int64_t)t * S + s;
    return contrib_val(oreT[i], metal[i], minedT[t], (int64_t)target[t], disc[t], pr, pc, mc, a, e,
                       sig ? sig[i] : 1.0);
}

struct ApplyArgs {
    Topo tp;
    int32_t S, S_pad, W, T, R, ore_off;
    uint32_t m_uniform;
    int32_t uniform;
    const uint32_t *mass;
    const float *val;
    const double *grade;
    uint32_t *blk;
    int64_t *minedT;
    int64_t *oreT;
    double *metal;
    double *npv;
    double *contrib;
    float *tab;
    const float4 *tabc;  // [T+1] Pout / Pin constants far from the target (uniform mass)
    float *ctab;  // nullptr when the period-pair table is not kept
    // FP32 shadow accumulators (precision study; nullptr when off): the same
    // per-period metal / contribution and NPV_s running totals kept in FP32
    float *metal32, *contrib32, *npv32;
    const double *disc;
    const double *sig;   // [T][S] uncertainty weights sigma(s,t) (Eq. 12); nullptr = none
    const uint64_t *cap;
    const uint64_t *target;
    double pr, pc, mc, a, e;
    ApplyResult *res;
    uint32_t *status;
};

// Sum over one warp of one FP64 value per lane (xor tree: every lane gets it).
static __device__ __forceinline__ double warp_sum_f64(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = __dadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// j-th block (0..21) whose lo/hi bounds a move of b1 (and b2) can change on the
// 1-5 grid: j = 11q + r, q = 0 for b1, 1 for b2; r = 0 the block itself,
// r = 1..10 the neighbour (dx, dy) of pattern entry (r - 1) / 2 one level up
// (r odd) or down (r even).  -1 when it does not exist.
static __device__ __forceinline__ int32_t apply_neighbour(const Topo &tp, int32_t b1, int32_t b2, int j) {
    const int32_t b = j < 11 ? b1 : b2;
    const int r = j < 11 ? j : j - 11;
    if (b < 0) return -1;
    if (r == 0) return b;
    const int32_t nxy = tp.nx * tp.ny;
    const int32_t x = b % tp.nx, y = (b / tp.nx) % tp.ny, z = b / nxy;
    const int k = (r - 1) >> 1;
    const int32_t px = x + (k == 1 ? -1 : (k == 2 ? 1 : 0)), py = y + (k == 3 ? -1 : (k == 4 ? 1 : 0));
    const int32_t pz = (r & 1) ? z - 1 : z + 1;
    if (px < 0 || px >= tp.nx || py < 0 || py >= tp.ny || pz < 0 || pz >= tp.nz) return -1;
    return px + tp.nx * (py + tp.ny * pz);
}

// Pout / Pin entries of period t, scenario s, for uniform block mass m from the
// excess x = oreT - Q_t.  Away from the target the entries do not depend on x:
// tc = (Pout for x >= m, Pout for x <= 0, Pin for x >= 0, Pin for x <= -m) holds
// the same FP64 expression evaluated at a representative x (same bits as
// table_entry); in between the expression is evaluated here.
static __device__ __forceinline__ void table_store_c(int t, int s, int32_t S_pad, int32_t T, int64_t x, float4 tc,
                                                     double d, int64_t m, double a, double e, float *tab,
                                                     float2 &out) {
    const float po = x >= m ? tc.x : (x <= 0 ? tc.y : __double2float_rn(__dmul_rn(d, pen_diff(x, x - m, a, e))));
    const float pi = x >= 0 ? tc.z : (x <= -m ? tc.w : __double2float_rn(__dmul_rn(d, pen_diff(x, x + m, a, e))));
    const int64_t io = (int64_t)t * S_pad + s;
    tab[io] = po;
    tab[(int64_t)(T + 1) * S_pad + io] = pi;
    out = make_float2(po, pi);
}

// Period-pair rows and columns of periods ra and rb (see apply_block), by
// worker w of nw (a warp each); tab and ctab do not overlap.
static __device__ __forceinline__ void ctab_rebuild(const float *__restrict__ tb, float *__restrict__ ct, uint32_t T1,
                                                    uint32_t S, size_t sp, uint32_t ra, uint32_t rb, int w, int nw,
                                                    int lane) {
    const uint32_t nsl = (S + 31) / 32;  // scenario slots of 32
    const uint32_t items = T1 * nsl;
    const size_t pin = (size_t)T1 * sp;
    for (uint32_t i0 = (uint32_t)w; i0 < items; i0 += 4u * (uint32_t)nw) {
        float pob[4], pib[4], poa[4], pia[4], por[4], pir[4];
        uint32_t bb[4], ss[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t it = i0 + (uint32_t)u * (uint32_t)nw;
            bb[u] = it / nsl;
            ss[u] = (it - bb[u] * nsl) * 32u + (uint32_t)lane;
            ok[u] = it < items && ss[u] < S;
            if (ok[u]) {
                pob[u] = tb[bb[u] * sp + ss[u]];
                pib[u] = tb[pin + bb[u] * sp + ss[u]];
                poa[u] = tb[ra * sp + ss[u]];
                pia[u] = tb[pin + ra * sp + ss[u]];
                por[u] = tb[rb * sp + ss[u]];
                pir[u] = tb[pin + rb * sp + ss[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (!ok[u]) continue;
            const uint32_t b = bb[u];
            const size_t s2 = ss[u];
            ct[((size_t)ra * T1 + b) * sp + s2] = poa[u] + pib[u];
            ct[((size_t)b * T1 + ra) * sp + s2] = pob[u] + pia[u];
            ct[((size_t)rb * T1 + b) * sp + s2] = por[u] + pib[u];
            ct[((size_t)b * T1 + rb) * sp + s2] = pob[u] + pir[u];
        }
    }
}

// Shared scratch of an apply: the new Pout / Pin entries of the two changed
// periods, 4 S_pad floats (S_pad <= 1024).
constexpr int kApplyTabMax = 4096;

// The FP64 side of scenario s's update for a move of b1 from t1 to t2 (and,
// for a swap, of b2 from t2 to t1): metal and discounted net cash of the two
// periods, and NPV_s; the FP32 shadow totals alongside when they are kept.
// nO1 / nO2 and mined1 / mined2 are the periods' ore and mined tonnage after
// the move; o1 / o2, gr1 / gr2 are the moved blocks' ore bits and grades in s;
// M, C and npv are the accumulators before the move.
static __device__ __forceinline__ void money_scenario(const ApplyArgs &A, int s, const MoveView &v, bool r1, bool r2,
                                                      uint32_t o1, uint32_t o2, double gr1, double gr2, int64_t nO1,
                                                      int64_t nO2, int64_t mined1, int64_t mined2, int64_t tgt1,
                                                      int64_t tgt2, double disc1, double disc2, double sg1, double sg2,
                                                      double M1, double M2, double C1, double C2, double my_npv) {
    const size_t i1 = (size_t)v.t1 * A.S + s, i2 = (size_t)v.t2 * A.S + s;
    const double g1 = o1 ? __dmul_rn((double)v.m1, gr1) : 0.0;
    const double g2 = (v.swap && o2) ? __dmul_rn((double)v.m2, gr2) : 0.0;
    double dnpv = 0.0;
    if (r1) {
        const double nM = __dadd_rn(__dsub_rn(M1, g1), g2);
        const double c = contrib_val(nO1, nM, mined1, tgt1, disc1, A.pr, A.pc, A.mc, A.a, A.e, sg1);
        dnpv = __dadd_rn(dnpv, __dsub_rn(c, C1));
        A.metal[i1] = nM;
        A.contrib[i1] = c;
    }
    if (r2) {
        const double nM = __dadd_rn(__dsub_rn(M2, g2), g1);
        const double c = contrib_val(nO2, nM, mined2, tgt2, disc2, A.pr, A.pc, A.mc, A.a, A.e, sg2);
        dnpv = __dadd_rn(dnpv, __dsub_rn(c, C2));
        A.metal[i2] = nM;
        A.contrib[i2] = c;
    }
    A.npv[s] = __dadd_rn(my_npv, dnpv);
    if (A.npv32) {
        // the same update with FP32 running totals
        float d32 = 0.0f;
        const float g1f = (float)g1, g2f = (float)g2;
        if (r1) {
            const float nM = A.metal32[i1] - g1f + g2f;
            const float c = contrib_val_f32(nO1, nM, mined1, tgt1, disc1, A.pr, A.pc, A.mc, A.a, A.e, sg1);
            d32 += c - A.contrib32[i1];
            A.metal32[i1] = nM;
            A.contrib32[i1] = c;
        }
        if (r2) {
            const float nM = A.metal32[i2] - g2f + g1f;
            const float c = contrib_val_f32(nO2, nM, mined2, tgt2, disc2, A.pr, A.pc, A.mc, A.a, A.e, sg2);
            d32 += c - A.contrib32[i2];
            A.metal32[i2] = nM;
            A.contrib32[i2] = c;
        }
        A.npv32[s] += d32;
    }
}

// Apply a decoded move v on a single CTA (blockDim.x >= max(S_pad, 64), a
// multiple of 32).  go = 1: v is valid, feasible and changes the schedule
// (the caller has checked it against the current state); go = 0: nothing
// changes.  MONEY = false does the structural part only (what the next
// evaluation reads: tonnage, schedule words, penalty tables); apply_money then
// does the FP64 part later, with the same arithmetic.  s_new: shared scratch
// of kApplyTabMax floats, 16-byte aligned.
//   1. one round trip of independent loads: per scenario (thread s) the moved
//      blocks' ore bits and the two affected periods' ore tonnage, mined
//      tonnage, target, discount (and for MONEY the grades, metal, NPV
//      contribution and NPV_s); the last warp the schedule words around the
//      moved blocks; every thread the Pout / Pin quads of the period-pair
//      items it rebuilds (when they are at most two per thread);
//   2. the last warp rewrites the packed period/lo/hi words of the moved
//      blocks and their grid neighbours (the moved blocks' new periods come
//      from the move, so the lanes need no ordering among themselves) while
//      thread s updates scenario s: ore tonnage and table entries of the two
//      periods, also kept in s_new (and for MONEY metal, contribution and
//      NPV_s += new - old); thread 0 the mined tonnage;
//   3. the threads rewrite the period-pair rows and columns of the two
//      periods, ctab[a][b] = Pout[a] + Pin[b], four scenarios per item.
// The NPV mean and std over scenarios are not formed here (k_npv_stats does
// that on request), so an apply ends with the state update.
template <bool MONEY>
static __device__ __forceinline__ void apply_core(const ApplyArgs &A, const MoveView &v, int go, float *s_new) {
    const int s = threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = blockDim.x, nwarp = nt >> 5;
    const bool hs = s < A.S;
    const uint32_t T = (uint32_t)A.T, T1 = T + 1;
    const size_t sp = (size_t)A.S_pad, pin = (size_t)T1 * sp;
    if (!go) return;
    const int32_t mb2 = v.swap ? v.b2 : -1;
    const bool r1 = v.t1 < T, r2 = v.t2 < T;
    const bool c1 = r1, c2 = r2 && v.t2 != v.t1;  // periods whose period-pair rows change
    const bool rebuild = A.ctab && A.uniform && (c1 || c2);
    const uint32_t qp = (uint32_t)(sp / 4), items = T1 * qp;
    const bool pre = rebuild && items <= 2u * (uint32_t)nt;  // the items' quads are loaded up front
    // 1. loads
    uint32_t o1 = 0, o2 = 0;
    double gr1 = 0.0, gr2 = 0.0, M1 = 0.0, M2 = 0.0, C1 = 0.0, C2 = 0.0, my_npv = 0.0, disc1 = 0.0, disc2 = 0.0;
    double sg1 = 1.0, sg2 = 1.0;
    int64_t O1 = 0, O2 = 0, tgt1 = 0, tgt2 = 0, mined1 = 0, mined2 = 0;
    float4 tc1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), tc2 = tc1;
    const size_t i1 = (size_t)v.t1 * A.S + s, i2 = (size_t)v.t2 * A.S + s;
    if (hs) {
        o1 = ore_bit(A.val, A.R, A.ore_off, v.b1, s);
        if (v.swap) o2 = ore_bit(A.val, A.R, A.ore_off, v.b2, s);
        if (MONEY) {
            gr1 = A.grade[(int64_t)v.b1 * A.S + s];
            if (v.swap) gr2 = A.grade[(int64_t)v.b2 * A.S + s];
            my_npv = A.npv[s];
        }
        if (r1) {
            O1 = A.oreT[i1];
            tgt1 = (int64_t)A.target[v.t1]; disc1 = A.disc[v.t1]; mined1 = A.minedT[v.t1];
            if (A.uniform) tc1 = A.tabc[v.t1];
            if (MONEY) {
                M1 = A.metal[i1]; C1 = A.contrib[i1];
                if (A.sig) sg1 = A.sig[i1];
            }
        }
        if (r2) {
            O2 = A.oreT[i2];
            tgt2 = (int64_t)A.target[v.t2]; disc2 = A.disc[v.t2]; mined2 = A.minedT[v.t2];
            if (A.uniform) tc2 = A.tabc[v.t2];
            if (MONEY) {
                M2 = A.metal[i2]; C2 = A.contrib[i2];
                if (A.sig) sg2 = A.sig[i2];
            }
        }
    }
    // the schedule words around the moved blocks (grid pattern): block j of
    // the last warp's lane and its ten grid neighbours, loaded together
    int32_t bj = -1;
    int32_t nb[10];
    uint32_t w[10], wj = 0u;
    if (A.tp.nx > 0 && warp == nwarp - 1 && lane < 22) {
        bj = apply_neighbour(A.tp, v.b1, mb2, lane);
        if (bj >= 0) {
            const int32_t nxy = A.tp.nx * A.tp.ny;
            const int32_t x = bj % A.tp.nx, y = (bj / A.tp.nx) % A.tp.ny, z = bj / nxy;
#pragma unroll
            for (int k = 0; k < 5; k++) {
                const int32_t px = x + (k == 1 ? -1 : (k == 2 ? 1 : 0)), py = y + (k == 3 ? -1 : (k == 4 ? 1 : 0));
                const bool in = px >= 0 && px < A.tp.nx && py >= 0 && py < A.tp.ny;
                nb[2 * k] = (in && z > 0) ? px + A.tp.nx * (py + A.tp.ny * (z - 1)) : -1;
                nb[2 * k + 1] = (in && z + 1 < A.tp.nz) ? px + A.tp.nx * (py + A.tp.ny * (z + 1)) : -1;
            }
#pragma unroll
            for (int k = 0; k < 10; k++) w[k] = nb[k] >= 0 ? A.blk[nb[k]] : 0u;
            wj = A.blk[bj];
        }
    }
    // Pout / Pin quads of the thread's period-pair items (b, q): it = s, s + nt
    const float4 *tb4 = reinterpret_cast<const float4 *>(A.tab);
    float4 pob[2], pib[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const uint32_t it = (uint32_t)s + (uint32_t)u * (uint32_t)nt;
        pob[u] = pib[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (pre && it < items) {
            pob[u] = tb4[it];              // item it = b * qp + q: Pout[b] quad q
            pib[u] = tb4[pin / 4 + it];    // Pin[b] quad q
        }
    }
    // 2. updates.  Every thread has read the mined tonnage of t1 and t2 above;
    // thread 0 overwrites it only after the barrier (go is uniform over the CTA)
    const int64_t dm1 = v.m1, dm2 = v.swap ? (int64_t)v.m2 : 0;
    mined1 += -dm1 + dm2;
    mined2 += dm1 - dm2;
    __syncthreads();
    if (threadIdx.x == 0) {  // thread 0 always holds a scenario (S >= 1), so it loaded both
        if (r1) A.minedT[v.t1] = mined1;
        if (r2) A.minedT[v.t2] = mined2;
    }
    // period of block j after the move: the moved blocks' from the move, the
    // others' from their words (of which only the lo/hi bits change here)
    auto period_after = [&](int32_t j) -> uint32_t {
        if (j == v.b1) return v.t2;
        if (j == mb2) return v.t1;
        return blk_period(A.blk[j]);
    };
    if (A.tp.nx > 0) {
        if (bj >= 0) {
            uint32_t lo = 0, hi = T;
#pragma unroll
            for (int k = 0; k < 10; k++) {
                if (nb[k] < 0) continue;
                const uint32_t t = nb[k] == v.b1 ? v.t2 : (nb[k] == mb2 ? v.t1 : blk_period(w[k]));
                if (k & 1) hi = t < hi ? t : hi;
                else lo = t > lo ? t : lo;
            }
            A.blk[bj] = blk_pack(bj == v.b1 ? v.t2 : (bj == mb2 ? v.t1 : blk_period(wj)), lo, hi);
        }
    } else {
        // CSR: the moved blocks and every direct predecessor and successor
        for (int q = 0; q < 2; q++) {
            const int32_t b = q == 0 ? v.b1 : mb2;
            if (b < 0) continue;
            const int32_t np = A.tp.pred_ptr[b + 1] - A.tp.pred_ptr[b];
            const int32_t ns = A.tp.succ_ptr[b + 1] - A.tp.succ_ptr[b];
            for (int k = threadIdx.x; k <= np + ns; k += blockDim.x) {
                const int32_t j = k == np + ns ? b
                                               : (k < np ? A.tp.pred_idx[A.tp.pred_ptr[b] + k]
                                                         : A.tp.succ_idx[A.tp.succ_ptr[b] + k - np]);
                A.blk[j] = block_bounds(A.tp, j, period_after);
            }
        }
    }
    float2 np1 = make_float2(0.0f, 0.0f), np2 = np1;  // new (Pout, Pin) of t1 and t2 (0 past S)
    if (hs) {
        const int64_t om1 = o1 ? (int64_t)v.m1 : 0, om2 = (v.swap && o2) ? (int64_t)v.m2 : 0;
        const int64_t nO1 = O1 + om2 - om1, nO2 = O2 + om1 - om2;
        const int64_t mu_ = (int64_t)A.m_uniform;
        if (r1) {
            A.oreT[i1] = nO1;
            if (A.uniform) table_store_c(v.t1, s, A.S_pad, A.T, nO1 - tgt1, tc1, disc1, mu_, A.a, A.e, A.tab, np1);
        }
        if (r2) {
            A.oreT[i2] = nO2;
            if (A.uniform) table_store_c(v.t2, s, A.S_pad, A.T, nO2 - tgt2, tc2, disc2, mu_, A.a, A.e, A.tab, np2);
        }
        if (MONEY)
            money_scenario(A, s, v, r1, r2, o1, o2, gr1, gr2, nO1, nO2, mined1, mined2, tgt1, tgt2, disc1, disc2,
                           sg1, sg2, M1, M2, C1, C2, my_npv);
    }
    if (!rebuild) return;
    const uint32_t ra = c1 ? v.t1 : v.t2, rb = c2 ? v.t2 : ra;
    if (!pre) {
        __syncthreads();  // the new Pout / Pin entries of t1 and t2 are in global memory
        ctab_rebuild(A.tab, A.ctab, T1, (uint32_t)A.S, sp, ra, rb, warp, nwarp, lane);
        return;
    }
    if ((size_t)s < sp) {  // s_new rows: Pout[t1], Pin[t1], Pout[t2], Pin[t2] after the move
        s_new[s] = np1.x;
        s_new[sp + s] = np1.y;
        s_new[2 * sp + s] = np2.x;
        s_new[3 * sp + s] = np2.y;
    }
    __syncthreads();
    // 3. ctab[a][b][s] = Pout[a][s] + Pin[b][s] for the rows a and columns b of
    // the changed periods, four scenarios per item; the new entries of t1 and
    // t2 come from s_new, every other operand was loaded in step 1
    const float4 *sn4 = reinterpret_cast<const float4 *>(s_new);
    auto po_new = [&](uint32_t t, uint32_t q) { return sn4[(t == v.t1 ? 0 : 2 * qp) + q]; };
    auto pi_new = [&](uint32_t t, uint32_t q) { return sn4[(t == v.t1 ? qp : 3 * qp) + q]; };
    float4 *ct4 = reinterpret_cast<float4 *>(A.ctab);
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const uint32_t it = (uint32_t)s + (uint32_t)u * (uint32_t)nt;
        if (it >= items) continue;
        const uint32_t b = it / qp, q = it - b * qp;
        const bool bnew = (c1 && b == v.t1) || (c2 && b == v.t2);
        const float4 pob_ = bnew ? po_new(b, q) : pob[u], pib_ = bnew ? pi_new(b, q) : pib[u];
        const float4 poa = po_new(ra, q), pia = pi_new(ra, q);
        const float4 por = po_new(rb, q), pir = pi_new(rb, q);
        ct4[((size_t)ra * T1 + b) * qp + q] = make_float4(poa.x + pib_.x, poa.y + pib_.y, poa.z + pib_.z, poa.w + pib_.w);
        ct4[((size_t)b * T1 + ra) * qp + q] = make_float4(pob_.x + pia.x, pob_.y + pia.y, pob_.z + pia.z, pob_.w + pia.w);
        ct4[((size_t)rb * T1 + b) * qp + q] = make_float4(por.x + pib_.x, por.y + pib_.y, por.z + pib_.z, por.w + pib_.w);
        ct4[((size_t)b * T1 + rb) * qp + q] = make_float4(pob_.x + pir.x, pob_.y + pir.y, pob_.z + pir.z, pob_.w + pir.w);
    }
}

// The FP64 part of an apply whose structural part (apply_core<false>) is done:
// info = (b1, b2 or B for a shift, t1 | t2 << 8, valid) of the move, uniform
// block mass.  The tonnage read here is the tonnage after the move, so the
// result is the same bits as a full apply.  The calling thread updates
// scenarios s_begin, s_begin + s_step, ... (scenarios are independent).
static __device__ __forceinline__ void apply_money(const ApplyArgs &A, int4 info, int s_begin, int s_step) {
    MoveView v;
    v.b1 = info.x;
    v.swap = info.y != A.tp.B;
    v.b2 = v.swap ? info.y : -1;
    v.t1 = (uint32_t)info.z & 0xffu;
    v.t2 = ((uint32_t)info.z >> 8) & 0xffu;
    v.m1 = A.m_uniform;
    v.m2 = v.swap ? A.m_uniform : 0u;
    const uint32_t T = (uint32_t)A.T;
    const bool r1 = v.t1 < T, r2 = v.t2 < T;
    for (int s = s_begin; s < A.S; s += s_step) {
        const size_t i1 = (size_t)v.t1 * A.S + s, i2 = (size_t)v.t2 * A.S + s;
        const uint32_t o1 = ore_bit(A.val, A.R, A.ore_off, v.b1, s);
        const uint32_t o2 = v.swap ? ore_bit(A.val, A.R, A.ore_off, v.b2, s) : 0u;
        const double gr1 = A.grade[(int64_t)v.b1 * A.S + s];
        const double gr2 = v.swap ? A.grade[(int64_t)v.b2 * A.S + s] : 0.0;
        int64_t nO1 = 0, nO2 = 0, mined1 = 0, mined2 = 0, tgt1 = 0, tgt2 = 0;
        double disc1 = 0.0, disc2 = 0.0, sg1 = 1.0, sg2 = 1.0, M1 = 0.0, M2 = 0.0, C1 = 0.0, C2 = 0.0;
        if (r1) {
            nO1 = A.oreT[i1]; mined1 = A.minedT[v.t1]; tgt1 = (int64_t)A.target[v.t1]; disc1 = A.disc[v.t1];
            M1 = A.metal[i1]; C1 = A.contrib[i1];
            if (A.sig) sg1 = A.sig[i1];
        }
        if (r2) {
            nO2 = A.oreT[i2]; mined2 = A.minedT[v.t2]; tgt2 = (int64_t)A.target[v.t2]; disc2 = A.disc[v.t2];
            M2 = A.metal[i2]; C2 = A.contrib[i2];
            if (A.sig) sg2 = A.sig[i2];
        }
        money_scenario(A, s, v, r1, r2, o1, o2, gr1, gr2, nO1, nO2, mined1, mined2, tgt1, tgt2, disc1, disc2, sg1,
                       sg2, M1, M2, C1, C2, A.npv[s]);
    }
}

// Apply one move on a single CTA (Algorithm 4: assign S[b*] <- t*): the moved
// blocks' schedule words, masses and the per-period tonnage and capacity are
// loaded, thread 0 re-checks the move exactly (decode_move) and records the
// outcome, then apply_core updates the state.  have = 0: nothing to apply.
static __device__ __noinline__ void apply_block(const ApplyArgs &A, int2 mv, int have, float *s_tab) {
    __shared__ MoveView sv;
    __shared__ int s_go;
    __shared__ int64_t s_mined[kMaxT + 1];
    __shared__ uint64_t s_cap[kMaxT + 1];
    __shared__ uint32_t s_w[2], s_m[2];
    const int32_t b1 = mv.x, b2 = mv.y;
    const bool ok1 = have && b1 >= 0 && b1 < A.tp.B;
    const bool ok2 = have && b2 >= 0 && b2 < A.tp.B;
    if (threadIdx.x == 0 && ok1) { s_w[0] = A.blk[b1]; s_m[0] = A.uniform ? A.m_uniform : A.mass[b1]; }
    if (threadIdx.x == 1 && ok2) { s_w[1] = A.blk[b2]; s_m[1] = A.uniform ? A.m_uniform : A.mass[b2]; }
    for (int t = threadIdx.x; t <= A.T; t += blockDim.x) {
        s_mined[t] = A.minedT[t];
        s_cap[t] = A.cap[t];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        MoveView v;
        if (have) {
            v = decode_move(
                mv, A.tp, [&](int32_t b) { return b == b1 ? s_w[0] : s_w[1]; },
                [&](int32_t b) { return b == b1 ? s_m[0] : s_m[1]; }, [&](uint32_t t) { return s_mined[t]; },
                [&](uint32_t t) { return s_cap[t]; });
        } else {
            v.valid = true;
            v.feasible = false;
            v.noop = true;
        }
        sv = v;
        s_go = have && v.valid && v.feasible && !v.noop;
        A.res->applied = (have && v.valid && v.feasible) ? 1 : 0;  // a feasible no-op counts as applied
        A.res->status = !have ? MM_OK : (!v.valid ? MM_ERR_BAD_MOVE : (!v.feasible ? MM_ERR_INFEASIBLE : MM_OK));
    }
    __syncthreads();
    const MoveView v = sv;
    apply_core<true>(A, v, s_go, s_tab);
}

// Apply a move that the same launch evaluated as feasible against the current
// state (the fused step's best move): no re-check is needed, so every load
// goes out at once.  info = (b1, b2 or B for a shift, t1 | t2 << 8) as the
// evaluator recorded it; have = 0: no feasible move.  Uniform block mass.
// MONEY = false: the structural part only (see apply_core).  Returns whether
// the state changed (a feasible move that is not a no-op).
template <bool MONEY>
static __device__ __noinline__ int apply_evaluated(const ApplyArgs &A, int4 info, int have, float *s_tab) {
    MoveView v;
    v.b1 = info.x;
    v.swap = info.y != A.tp.B;
    v.b2 = v.swap ? info.y : -1;
    v.t1 = (uint32_t)info.z & 0xffu;
    v.t2 = ((uint32_t)info.z >> 8) & 0xffu;
    v.m1 = A.m_uniform;
    v.m2 = v.swap ? A.m_uniform : 0u;
    v.valid = true;
    v.feasible = true;
    v.noop = v.swap ? (v.b1 == v.b2 || v.t1 == v.t2) : v.t1 == v.t2;
    if (threadIdx.x == 0) {
        A.res->applied = have ? 1 : 0;
        A.res->status = MM_OK;
    }
    apply_core<MONEY>(A, v, have && !v.noop, s_tab);
    return have && !v.noop;
}

}  // namespace mm
