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

// Pout/Pin entry of period t, scenario s from its excess x = oreT - Q_t (t < T, s < S).
__device__ __forceinline__ void table_store(int t, int s, int32_t S_pad, int32_t T, int64_t x, double d, int64_t m,
                                            double a, double e, float *tab) {
    tab[(int64_t)t * S_pad + s] = __double2float_rn(__dmul_rn(d, pen_diff(x, x - m, a, e)));
    tab[(int64_t)(T + 1) * S_pad + (int64_t)t * S_pad + s] = __double2float_rn(__dmul_rn(d, pen_diff(x, x + m, a, e)));
}

// Discounted net cash of a period from its accumulators (pure form):
//   d_t (price*rec*metal - pc*ore_t - mc*mined_t - pen_t(ore_t)).
__device__ __forceinline__ double contrib_val(int64_t o, double metal, int64_t mined, int64_t target, double disc,
                                              double pr, double pc, double mc, double a, double e) {
    double cash = __dsub_rn(__dsub_rn(__dmul_rn(pr, metal), __dmul_rn(pc, (double)o)), __dmul_rn(mc, (double)mined));
    return __dmul_rn(disc, __dsub_rn(cash, pen_of(o - target, a, e)));
}

// contrib_val in FP32 throughout (the FP32 shadow accumulators).
__device__ __forceinline__ float contrib_val_f32(int64_t o, float metal, int64_t mined, int64_t target, double disc,
                                                double pr, double pc, double mc, double a, double e) {
    const float of = (float)o, dev = (float)(o - target);
    const float cash = (float)pr * metal - (float)pc * of - (float)mc * (float)mined;
    const float pen = dev < 0.0f ? (float)a * -dev : (float)e * dev;
    return (float)disc * (cash - pen);
}

// Discounted net cash of period t in scenario s:
//   d_t (price*rec*metal - pc*oreT - mc*minedT - pen_t(oreT)).
__device__ __forceinline__ double contrib_of(int t, int s, int32_t S, const double *disc, const double *metal,
                                             const int64_t *oreT, const int64_t *minedT, const uint64_t *target,
                                             double pr, double pc, double mc, double a, double e) {
    int64_t o = oreT[(int64_t)t * S + s];
    double cash = __dsub_rn(__dsub_rn(__dmul_rn(pr, metal[(int64_t)t * S + s]), __dmul_rn(pc, (double)o)),
                            __dmul_rn(mc, (double)minedT[t]));
    double p = pen_of(o - (int64_t)target[t], a, e);
    return __dmul_rn(disc[t], __dsub_rn(cash, p));
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
    float *ctab;  // nullptr when the period-pair table is not kept
    // FP32 shadow accumulators (precision study; nullptr when off): the same
    // per-period metal / contribution and NPV_s running totals kept in FP32
    float *metal32, *contrib32, *npv32;
    const double *disc;
    const uint64_t *cap;
    const uint64_t *target;
    double pr, pc, mc, a, e;
    ApplyResult *res;
    uint32_t *status;
};

// Apply one move on a single CTA: exact re-check, period update, integer
// tonnages, FP64 metal, lo/hi of the neighbourhood, tables and NPV
// contributions of the affected periods (NPV_s += new - old), then the FP64
// mean/std of NPV over scenarios (computed whether or not the move applied).
// The move comes either by value (from_dev = 0) or as moves[idx[0]] when
// *count > 0 (from_dev = 1).
// Sum over the block of one FP64 value per thread, where only threads s < n
// hold values: only the warps holding values reduce (FP64 is scarce on this
// part), and thread 0 combines their partials.  Result valid in thread 0.
static __device__ __forceinline__ double block_sum_f64(double x, int n, double *red) {
    const int nwv = (n + 31) >> 5;  // warps holding values
    const int warp = threadIdx.x >> 5;
    if (warp < nwv) {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[warp] = x;
    }
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nwv; w++) t += red[w];
    __syncthreads();
    return t;
}

// The whole CTA applies one move (blockDim.x >= S; any block size from 64):
//   1. one round trip of independent loads: the moved blocks' schedule words
//      and masses, every period's tonnage and capacity, and per scenario
//      (thread s) the moved blocks' ore bits and FP64 grades;
//   2. thread 0 re-checks the move exactly and updates periods and tonnage;
//   3. per scenario: the two affected periods' ore tonnage, metal, NPV
//      contribution and table entries (NPV_s += new - old), and the lo/hi
//      bounds of the moved blocks' neighbourhood;
//   4. FP64 mean and population std of NPV over scenarios, computed whether
//      or not the move applied.
// have = 0: nothing to apply (statistics only).
static __device__ __noinline__ void apply_block(const ApplyArgs &A, int2 mv, int have) {
    __shared__ MoveView sv;
    __shared__ int s_go;
    __shared__ int32_t s_nb[32];
    __shared__ int s_nnb;
    __shared__ int64_t s_mined[kMaxT + 1];
    __shared__ uint64_t s_cap[kMaxT + 1];
    __shared__ uint32_t s_w[2], s_m[2];
    __shared__ double red[33];
    const int s = threadIdx.x;
    const bool hs = s < A.S;
    const int32_t b1 = mv.x, b2 = mv.y;
    const bool ok1 = have && b1 >= 0 && b1 < A.tp.B;
    const bool ok2 = have && b2 >= 0 && b2 < A.tp.B;
    // 1. independent loads
    if (threadIdx.x == 0 && ok1) { s_w[0] = A.blk[b1]; s_m[0] = A.uniform ? A.m_uniform : A.mass[b1]; }
    if (threadIdx.x == 1 && ok2) { s_w[1] = A.blk[b2]; s_m[1] = A.uniform ? A.m_uniform : A.mass[b2]; }
    for (int t = threadIdx.x; t <= A.T; t += blockDim.x) {
        s_mined[t] = A.minedT[t];
        s_cap[t] = A.cap[t];
    }
    const uint32_t o1 = (hs && ok1) ? ore_bit(A.val, A.R, A.ore_off, b1, s) : 0u;
    const uint32_t o2 = (hs && ok2) ? ore_bit(A.val, A.R, A.ore_off, b2, s) : 0u;
    const double gr1 = (hs && ok1) ? A.grade[(int64_t)b1 * A.S + s] : 0.0;
    const double gr2 = (hs && ok2) ? A.grade[(int64_t)b2 * A.S + s] : 0.0;
    __syncthreads();
    // 2. exact re-check and the scalar updates
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
        const int go = have && v.valid && v.feasible && !v.noop;
        s_go = go;
        A.res->applied = (have && v.valid && v.feasible) ? 1 : 0;  // a feasible no-op counts as applied
        A.res->status = !have ? MM_OK : (!v.valid ? MM_ERR_BAD_MOVE : (!v.feasible ? MM_ERR_INFEASIBLE : MM_OK));
        if (go) {
            const int64_t dm1 = v.m1, dm2 = v.swap ? (int64_t)v.m2 : 0;
            if (v.t1 < (uint32_t)A.T) A.minedT[v.t1] = (s_mined[v.t1] += -dm1 + dm2);
            if (v.t2 < (uint32_t)A.T) A.minedT[v.t2] = (s_mined[v.t2] += dm1 - dm2);
            A.blk[v.b1] = (s_w[0] & ~0xffu) | v.t2;  // lo/hi are recomputed below
            if (v.swap) A.blk[v.b2] = (s_w[1] & ~0xffu) | v.t1;
            // neighbourhood whose lo/hi may change: moved blocks and their neighbours
            int n = 0;
            const int32_t mb[2] = {v.b1, v.swap ? v.b2 : -1};
            for (int q = 0; q < 2; q++) {
                const int32_t b = mb[q];
                if (b < 0) continue;
                s_nb[n++] = b;
                if (A.tp.nx > 0) {
                    const int32_t nxy = A.tp.nx * A.tp.ny;
                    const int32_t x = b % A.tp.nx, y = (b / A.tp.nx) % A.tp.ny, z = b / nxy;
                    const int dx[5] = {0, -1, 1, 0, 0};
                    const int dy[5] = {0, 0, 0, -1, 1};
                    for (int k = 0; k < 5; k++) {
                        const int32_t px = x + dx[k], py = y + dy[k];
                        if (px < 0 || px >= A.tp.nx || py < 0 || py >= A.tp.ny) continue;
                        if (z > 0) s_nb[n++] = px + A.tp.nx * (py + A.tp.ny * (z - 1));
                        if (z + 1 < A.tp.nz) s_nb[n++] = px + A.tp.nx * (py + A.tp.ny * (z + 1));
                    }
                }
            }
            s_nnb = n;
        }
    }
    __syncthreads();
    // 3. per-scenario updates of the two affected periods
    double my_npv = hs ? A.npv[s] : 0.0;
    if (s_go) {
        const MoveView v = sv;
        if (A.tp.nx > 0 && threadIdx.x < (unsigned)s_nnb) {
            const int32_t b = s_nb[threadIdx.x];
            A.blk[b] = block_bounds(A.tp, b, [&](int32_t j) { return blk_period(A.blk[j]); });
        }
        if (hs) {
            const bool r1 = v.t1 < (uint32_t)A.T, r2 = v.t2 < (uint32_t)A.T;
            const size_t i1 = (size_t)v.t1 * A.S + s, i2 = (size_t)v.t2 * A.S + s;
            const int64_t O1 = r1 ? A.oreT[i1] : 0, O2 = r2 ? A.oreT[i2] : 0;
            const double M1 = r1 ? A.metal[i1] : 0.0, M2 = r2 ? A.metal[i2] : 0.0;
            const double C1 = r1 ? A.contrib[i1] : 0.0, C2 = r2 ? A.contrib[i2] : 0.0;
            const int64_t tgt1 = r1 ? (int64_t)A.target[v.t1] : 0, tgt2 = r2 ? (int64_t)A.target[v.t2] : 0;
            const double disc1 = r1 ? A.disc[v.t1] : 0.0, disc2 = r2 ? A.disc[v.t2] : 0.0;
            const int64_t mined1 = r1 ? s_mined[v.t1] : 0, mined2 = r2 ? s_mined[v.t2] : 0;
            const int64_t om1 = o1 ? (int64_t)v.m1 : 0, om2 = (v.swap && o2) ? (int64_t)v.m2 : 0;
            const double g1 = o1 ? __dmul_rn((double)v.m1, gr1) : 0.0;
            const double g2 = (v.swap && o2) ? __dmul_rn((double)v.m2, gr2) : 0.0;
            const int64_t mu_ = (int64_t)A.m_uniform;
            double dnpv = 0.0;
            if (r1) {
                const int64_t nO = O1 + om2 - om1;
                const double nM = __dadd_rn(__dsub_rn(M1, g1), g2);
                const double c = contrib_val(nO, nM, mined1, tgt1, disc1, A.pr, A.pc, A.mc, A.a, A.e);
                dnpv = __dadd_rn(dnpv, __dsub_rn(c, C1));
                A.oreT[i1] = nO;
                A.metal[i1] = nM;
                A.contrib[i1] = c;
                if (A.uniform) table_store(v.t1, s, A.S_pad, A.T, nO - tgt1, disc1, mu_, A.a, A.e, A.tab);
            }
            if (r2) {
                const int64_t nO = O2 + om1 - om2;
                const double nM = __dadd_rn(__dsub_rn(M2, g2), g1);
                const double c = contrib_val(nO, nM, mined2, tgt2, disc2, A.pr, A.pc, A.mc, A.a, A.e);
                dnpv = __dadd_rn(dnpv, __dsub_rn(c, C2));
                A.oreT[i2] = nO;
                A.metal[i2] = nM;
                A.contrib[i2] = c;
                if (A.uniform) table_store(v.t2, s, A.S_pad, A.T, nO - tgt2, disc2, mu_, A.a, A.e, A.tab);
            }
            my_npv = __dadd_rn(my_npv, dnpv);
            A.npv[s] = my_npv;
            if (A.npv32) {
                // the same update with FP32 running totals
                float d32 = 0.0f;
                const float g1f = (float)g1, g2f = (float)g2;
                if (r1) {
                    const float nM = A.metal32[i1] - g1f + g2f;
                    const float c = contrib_val_f32(O1 + om2 - om1, nM, mined1, tgt1, disc1, A.pr, A.pc, A.mc, A.a, A.e);
                    d32 += c - A.contrib32[i1];
                    A.metal32[i1] = nM;
                    A.contrib32[i1] = c;
                }
                if (r2) {
                    const float nM = A.metal32[i2] - g2f + g1f;
                    const float c = contrib_val_f32(O2 + om1 - om2, nM, mined2, tgt2, disc2, A.pr, A.pc, A.mc, A.a, A.e);
                    d32 += c - A.contrib32[i2];
                    A.metal32[i2] = nM;
                    A.contrib32[i2] = c;
                }
                A.npv32[s] += d32;
            }
        }
        if (A.ctab) {
            // period-pair table: rows and columns of the changed periods
            __syncthreads();  // the new Pout / Pin entries of t1 and t2 are written
            const uint32_t T = (uint32_t)A.T, T1 = T + 1;
            const bool c1 = v.t1 < T, c2 = v.t2 < T && v.t2 != v.t1;
            if (c1 || c2) {
                const uint32_t ra = c1 ? v.t1 : v.t2, rb = c2 ? v.t2 : ra;
                const size_t sp = (size_t)A.S_pad, pin = (size_t)T1 * sp;
                const float *tb = A.tab;
                for (int j = threadIdx.x; j < (int)T1 * A.S; j += blockDim.x) {
                    const uint32_t b = (uint32_t)(j / A.S), s2 = (uint32_t)(j - (int)b * A.S);
                    const float pob = tb[b * sp + s2], pib = tb[pin + b * sp + s2];
                    const float poa = tb[ra * sp + s2], pia = tb[pin + ra * sp + s2];
                    const float por = tb[rb * sp + s2], pir = tb[pin + rb * sp + s2];
                    A.ctab[((size_t)ra * T1 + b) * sp + s2] = poa + pib;
                    A.ctab[((size_t)b * T1 + ra) * sp + s2] = pob + pia;
                    A.ctab[((size_t)rb * T1 + b) * sp + s2] = por + pib;
                    A.ctab[((size_t)b * T1 + rb) * sp + s2] = pob + pir;
                }
            }
        }
        if (A.tp.nx == 0) {
            // CSR: the moved blocks first, then every predecessor and successor
            if (threadIdx.x < 2) {
                const int32_t b = threadIdx.x == 0 ? v.b1 : (v.swap ? v.b2 : -1);
                if (b >= 0) A.blk[b] = block_bounds(A.tp, b, [&](int32_t j) { return blk_period(A.blk[j]); });
            }
            __syncthreads();
            for (int q = 0; q < 2; q++) {
                const int32_t b = q == 0 ? v.b1 : (v.swap ? v.b2 : -1);
                if (b < 0) continue;
                const int32_t np = A.tp.pred_ptr[b + 1] - A.tp.pred_ptr[b];
                const int32_t ns = A.tp.succ_ptr[b + 1] - A.tp.succ_ptr[b];
                for (int k = threadIdx.x; k < np + ns; k += blockDim.x) {
                    const int32_t j = k < np ? A.tp.pred_idx[A.tp.pred_ptr[b] + k] : A.tp.succ_idx[A.tp.succ_ptr[b] + k - np];
                    A.blk[j] = block_bounds(A.tp, j, [&](int32_t i) { return blk_period(A.blk[i]); });
                }
                __syncthreads();
            }
        }
    }
    // 4. statistics (two passes, values in registers; thread 0 divides)
    const double sum = block_sum_f64(my_npv, A.S, red);
    if (threadIdx.x == 0) red[32] = sum / A.S;
    __syncthreads();
    const double mean = red[32];
    const double dv = hs ? my_npv - mean : 0.0;
    const double ss = block_sum_f64(dv * dv, A.S, red);
    if (threadIdx.x == 0) {
        A.res->mean = mean;
        A.res->std = sqrt(ss / A.S);
    }
}

}  // namespace mm
