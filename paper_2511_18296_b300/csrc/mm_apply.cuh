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

// Shared-memory copy of the Pout / Pin tables used by the period-pair rebuild
// when 2 (T+1) S_pad floats fit (18 KB).
constexpr int kApplyTabMax = 4608;

// Apply a decoded move v on a single CTA (blockDim.x >= max(S, 64), a multiple
// of 32).  go = 1: v is valid, feasible and changes the schedule (the caller
// has checked it against the current state); go = 0: nothing changes.
//   1. one round trip of independent loads: per scenario (thread s) the moved
//      blocks' ore bits and FP64 grades and the two affected periods' ore
//      tonnage, metal, NPV contribution, mined tonnage, target and discount;
//      the Pout / Pin tables into shared memory where they fit;
//   2. the last warp rewrites the packed period/lo/hi words of the moved
//      blocks and their grid neighbours (the moved blocks' new periods come
//      from the move, so the lanes need no ordering among themselves) while
//      thread s updates scenario s: ore tonnage, metal, NPV contribution and
//      table entries of the two periods (NPV_s += new - old); thread 0 the
//      mined tonnage;
//   3. the warps rebuild the period-pair rows and columns of the two periods.
// The NPV mean and std over scenarios are not formed here (k_npv_stats does
// that on request), so an apply ends with the state update.
static __device__ __forceinline__ void apply_core(const ApplyArgs &A, const MoveView &v, int go) {
    __shared__ __align__(16) float s_tab[kApplyTabMax];
    const int s = threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    const bool hs = s < A.S;
    const uint32_t T = (uint32_t)A.T, T1 = T + 1;
    const size_t sp = (size_t)A.S_pad, pin = (size_t)T1 * sp;
    const bool tab_sm = A.ctab && 2 * pin <= (size_t)kApplyTabMax;
    if (!go) return;
    const int32_t mb2 = v.swap ? v.b2 : -1;
    const bool r1 = v.t1 < T, r2 = v.t2 < T;
    const bool c1 = r1, c2 = r2 && v.t2 != v.t1;  // periods whose period-pair rows change
    const bool stage = tab_sm && (c1 || c2);     // copies issued here are always waited for below
    // 1. loads: the Pout / Pin tables go to shared memory by asynchronous
    // 16-byte copies, all in flight at once (waited for before the rebuild)
    if (stage) {
        const uint32_t n16 = (uint32_t)(2 * pin / 4);
        for (uint32_t i = threadIdx.x; i < n16; i += blockDim.x)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(s_tab + 4 * i)),
                         "l"(A.tab + 4 * (size_t)i)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    uint32_t o1 = 0, o2 = 0;
    double gr1 = 0.0, gr2 = 0.0, M1 = 0.0, M2 = 0.0, C1 = 0.0, C2 = 0.0, my_npv = 0.0, disc1 = 0.0, disc2 = 0.0;
    double sg1 = 1.0, sg2 = 1.0;
    int64_t O1 = 0, O2 = 0, tgt1 = 0, tgt2 = 0, mined1 = 0, mined2 = 0;
    float4 tc1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), tc2 = tc1;
    const size_t i1 = (size_t)v.t1 * A.S + s, i2 = (size_t)v.t2 * A.S + s;
    if (hs) {
        o1 = ore_bit(A.val, A.R, A.ore_off, v.b1, s);
        gr1 = A.grade[(int64_t)v.b1 * A.S + s];
        if (v.swap) {
            o2 = ore_bit(A.val, A.R, A.ore_off, v.b2, s);
            gr2 = A.grade[(int64_t)v.b2 * A.S + s];
        }
        my_npv = A.npv[s];
        if (r1) {
            O1 = A.oreT[i1]; M1 = A.metal[i1]; C1 = A.contrib[i1];
            tgt1 = (int64_t)A.target[v.t1]; disc1 = A.disc[v.t1]; mined1 = A.minedT[v.t1];
            if (A.sig) sg1 = A.sig[i1];
            if (A.uniform) tc1 = A.tabc[v.t1];
        }
        if (r2) {
            O2 = A.oreT[i2]; M2 = A.metal[i2]; C2 = A.contrib[i2];
            tgt2 = (int64_t)A.target[v.t2]; disc2 = A.disc[v.t2]; mined2 = A.minedT[v.t2];
            if (A.sig) sg2 = A.sig[i2];
            if (A.uniform) tc2 = A.tabc[v.t2];
        }
    }
    // 2. updates.  Every thread has read the mined tonnage of t1 and t2 above;
    // thread 0 overwrites it only after the barrier (go is uniform over the CTA)
    const int64_t dm1 = v.m1, dm2 = v.swap ? (int64_t)v.m2 : 0;
    mined1 += -dm1 + dm2;
    mined2 += dm1 - dm2;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (r1) A.minedT[v.t1] = A.minedT[v.t1] - dm1 + dm2;
        if (r2) A.minedT[v.t2] = A.minedT[v.t2] + dm1 - dm2;
    }
    // period of block j after the move: the moved blocks' from the move, the
    // others' from their words (of which only the lo/hi bits change here)
    auto period_after = [&](int32_t j) -> uint32_t {
        if (j == v.b1) return v.t2;
        if (j == mb2) return v.t1;
        return blk_period(A.blk[j]);
    };
    if (A.tp.nx > 0) {
        if (warp == nwarp - 1 && lane < 22) {
            const int32_t b = apply_neighbour(A.tp, v.b1, mb2, lane);
            if (b >= 0) {
                // the ten grid neighbours' words are loaded together, then the
                // moved blocks' periods are substituted
                const int32_t nxy = A.tp.nx * A.tp.ny;
                const int32_t x = b % A.tp.nx, y = (b / A.tp.nx) % A.tp.ny, z = b / nxy;
                int32_t nb[10];
                uint32_t w[10];
#pragma unroll
                for (int k = 0; k < 5; k++) {
                    const int32_t px = x + (k == 1 ? -1 : (k == 2 ? 1 : 0)), py = y + (k == 3 ? -1 : (k == 4 ? 1 : 0));
                    const bool in = px >= 0 && px < A.tp.nx && py >= 0 && py < A.tp.ny;
                    nb[2 * k] = (in && z > 0) ? px + A.tp.nx * (py + A.tp.ny * (z - 1)) : -1;
                    nb[2 * k + 1] = (in && z + 1 < A.tp.nz) ? px + A.tp.nx * (py + A.tp.ny * (z + 1)) : -1;
                }
#pragma unroll
                for (int k = 0; k < 10; k++) w[k] = nb[k] >= 0 ? A.blk[nb[k]] : 0u;
                uint32_t lo = 0, hi = T;
#pragma unroll
                for (int k = 0; k < 10; k++) {
                    if (nb[k] < 0) continue;
                    const uint32_t t = nb[k] == v.b1 ? v.t2 : (nb[k] == mb2 ? v.t1 : blk_period(w[k]));
                    if (k & 1) hi = t < hi ? t : hi;
                    else lo = t > lo ? t : lo;
                }
                A.blk[b] = blk_pack(b == v.b1 ? v.t2 : (b == mb2 ? v.t1 : blk_period(A.blk[b])), lo, hi);
            }
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
    float2 np1 = make_float2(0.0f, 0.0f), np2 = np1;  // new (Pout, Pin) of t1 and t2
    if (hs) {
        const int64_t om1 = o1 ? (int64_t)v.m1 : 0, om2 = (v.swap && o2) ? (int64_t)v.m2 : 0;
        const double g1 = o1 ? __dmul_rn((double)v.m1, gr1) : 0.0;
        const double g2 = (v.swap && o2) ? __dmul_rn((double)v.m2, gr2) : 0.0;
        const int64_t mu_ = (int64_t)A.m_uniform;
        double dnpv = 0.0;
        if (r1) {
            const int64_t nO = O1 + om2 - om1;
            const double nM = __dadd_rn(__dsub_rn(M1, g1), g2);
            const double c = contrib_val(nO, nM, mined1, tgt1, disc1, A.pr, A.pc, A.mc, A.a, A.e, sg1);
            dnpv = __dadd_rn(dnpv, __dsub_rn(c, C1));
            A.oreT[i1] = nO;
            A.metal[i1] = nM;
            A.contrib[i1] = c;
            if (A.uniform) table_store_c(v.t1, s, A.S_pad, A.T, nO - tgt1, tc1, disc1, mu_, A.a, A.e, A.tab, np1);
        }
        if (r2) {
            const int64_t nO = O2 + om1 - om2;
            const double nM = __dadd_rn(__dsub_rn(M2, g2), g1);
            const double c = contrib_val(nO, nM, mined2, tgt2, disc2, A.pr, A.pc, A.mc, A.a, A.e, sg2);
            dnpv = __dadd_rn(dnpv, __dsub_rn(c, C2));
            A.oreT[i2] = nO;
            A.metal[i2] = nM;
            A.contrib[i2] = c;
            if (A.uniform) table_store_c(v.t2, s, A.S_pad, A.T, nO - tgt2, tc2, disc2, mu_, A.a, A.e, A.tab, np2);
        }
        my_npv = __dadd_rn(my_npv, dnpv);
        A.npv[s] = my_npv;
        if (A.npv32) {
            // the same update with FP32 running totals
            float d32 = 0.0f;
            const float g1f = (float)g1, g2f = (float)g2;
            if (r1) {
                const float nM = A.metal32[i1] - g1f + g2f;
                const float c = contrib_val_f32(O1 + om2 - om1, nM, mined1, tgt1, disc1, A.pr, A.pc, A.mc, A.a, A.e, sg1);
                d32 += c - A.contrib32[i1];
                A.metal32[i1] = nM;
                A.contrib32[i1] = c;
            }
            if (r2) {
                const float nM = A.metal32[i2] - g2f + g1f;
                const float c = contrib_val_f32(O2 + om1 - om2, nM, mined2, tgt2, disc2, A.pr, A.pc, A.mc, A.a, A.e, sg2);
                d32 += c - A.contrib32[i2];
                A.metal32[i2] = nM;
                A.contrib32[i2] = c;
            }
            A.npv32[s] += d32;
        }
    }
    if (!A.ctab || !(c1 || c2)) return;
    const uint32_t ra = c1 ? v.t1 : v.t2, rb = c2 ? v.t2 : ra;
    if (!tab_sm) {
        __syncthreads();  // the new Pout / Pin entries of t1 and t2 are in global memory
        ctab_rebuild(A.tab, A.ctab, T1, (uint32_t)A.S, sp, ra, rb, warp, nwarp, lane);
        return;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();  // every staged row has landed
    if (hs && A.uniform) {
        if (r1) { s_tab[v.t1 * sp + s] = np1.x; s_tab[pin + v.t1 * sp + s] = np1.y; }
        if (r2) { s_tab[v.t2 * sp + s] = np2.x; s_tab[pin + v.t2 * sp + s] = np2.y; }
    }
    __syncthreads();
    // 3. ctab[a][b][s] = Pout[a][s] + Pin[b][s] for the rows a and columns b of
    // the changed periods, four scenarios per item, every operand in shared
    // memory: only the 16-byte stores leave the SM
    const uint32_t qp = (uint32_t)(sp / 4), items = T1 * qp;
    const float4 *st4 = reinterpret_cast<const float4 *>(s_tab);
    float4 *ct4 = reinterpret_cast<float4 *>(A.ctab);
    const size_t pin4 = (size_t)T1 * qp;
    for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
        const uint32_t b = it / qp, q = it - b * qp;
        const float4 pob = st4[b * qp + q], pib = st4[pin4 + b * qp + q];
        const float4 poa = st4[ra * qp + q], pia = st4[pin4 + ra * qp + q];
        const float4 por = st4[rb * qp + q], pir = st4[pin4 + rb * qp + q];
        ct4[((size_t)ra * T1 + b) * qp + q] = make_float4(poa.x + pib.x, poa.y + pib.y, poa.z + pib.z, poa.w + pib.w);
        ct4[((size_t)b * T1 + ra) * qp + q] = make_float4(pob.x + pia.x, pob.y + pia.y, pob.z + pia.z, pob.w + pia.w);
        ct4[((size_t)rb * T1 + b) * qp + q] = make_float4(por.x + pib.x, por.y + pib.y, por.z + pib.z, por.w + pib.w);
        ct4[((size_t)b * T1 + rb) * qp + q] = make_float4(pob.x + pir.x, pob.y + pir.y, pob.z + pir.z, pob.w + pir.w);
    }
}

// Apply one move on a single CTA (Algorithm 4: assign S[b*] <- t*): the moved
// blocks' schedule words, masses and the per-period tonnage and capacity are
// loaded, thread 0 re-checks the move exactly (decode_move) and records the
// outcome, then apply_core updates the state.  have = 0: nothing to apply.
static __device__ __noinline__ void apply_block(const ApplyArgs &A, int2 mv, int have) {
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
    apply_core(A, v, s_go);
}

// Apply a move that the same launch evaluated as feasible against the current
// state (the fused step's best move): no re-check is needed, so every load
// goes out at once.  info = (b1, b2 or B for a shift, t1 | t2 << 8) as the
// evaluator recorded it; have = 0: no feasible move.  Uniform block mass.
static __device__ __noinline__ void apply_evaluated(const ApplyArgs &A, int4 info, int have) {
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
    apply_core(A, v, have && !v.noop);
}

}  // namespace mm
