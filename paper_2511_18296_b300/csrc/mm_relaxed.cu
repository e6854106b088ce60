// Relaxed objective: forward and hand-written adjoint.
//
// The extraction decision x[b][t] of Eq. 14 relaxed to [0, 1], the mill
// penalty smoothed by a softplus of width m_ref / beta, and the risk term
// J = mean_s NPV_s - lambda std_s NPV_s:
//   O[t][s] = sum_b x[b][t] m_b ore[b][s],   V[t][s] = sum_b x[b][t] v[b][s],
//   NPV_s   = sum_t d_t (V[t][s] - P_t(O[t][s])),
//   P_t(O)  = a m_ref sp((Q_t - O) / m_ref) + e m_ref sp((O - Q_t) / m_ref),
//   sp(z)   = log(1 + exp(beta z)) / beta.
// ore and v come from the grades g exactly as in the discrete model; ore is a
// step in g and carries no gradient.  With the model's own grades the model's
// ore bits and FP32 value rows are read.  With caller grades (FP32) the FP64
// ore decision ((g price) recovery > pc) is monotone in g when price and
// recovery are positive and pc is not negative, so it equals g >= g_t for one
// float g_t, found on the host with the same FP64 expression: the kernels
// compare in FP32 and take identical decisions (FP64 runs at a small fraction
// of the FP32 rate on this part); otherwise they evaluate the FP64 test.
//
// Forward: the two skinny contractions over blocks run on CUDA cores -- each
// CTA takes a chunk of blocks and a tile of periods, one thread per scenario,
// FP32 products summed over the chunk -- and the chunk partials are added in
// FP64 in chunk order (deterministic), one warp per (t, s).  O[t][s] is kept as
// the checkpoint the adjoint reads, so the backward pass never redoes the
// contraction.  The smoothed penalty and its derivative evaluate the
// exponential and logarithm in FP32 on an argument formed in FP64.
// Adjoint: with w_s = dJ/dNPV_s and c[t][s] = w_s P_t'(O[t][s]),
//   dJ/dx[b][t] = d_t (sum_s w_s v[b][s] - m_b sum_s c[t][s] ore[b][s]),
//   dJ/dg[b][s] = w_s ore[b][s] m_b price recovery sum_t d_t x[b][t],
// one warp per block.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mm_internal.cuh"

namespace mm {

constexpr int kRelaxTile = 24;    // periods per forward CTA (at most)

struct RelaxEcon {
    double p, r, pc;   // price, recovery, processing cost (FP64 ore decision)
    float pf, rf, pcf, mcf;
    double a, e, lambda, beta, m_ref;
    double inv_beta, inv_mref, inv_S;  // reciprocals formed on the host (FP64 division is slow on this part)
    float g_thr;       // ore iff g >= g_thr, when use_thr
    int32_t use_thr;
};

// Model rows (values, then ore words) for the model-grade path.
struct RelaxRows {
    const float *val;
    int32_t R, ore_off;
};

template <typename G>
__device__ __forceinline__ bool relax_ore(G g, const RelaxEcon &E) {
    if (E.use_thr) return (float)g >= E.g_thr;
    return ((double)g * E.p) * E.r > E.pc;
}

// ore and v of (b, s): from the model's rows (model grades) or the grade.
template <typename G>
__device__ __forceinline__ void relax_ore_value(const G *g, const RelaxRows &Rw, int32_t b, int32_t S, int s, float m,
                                                const RelaxEcon &E, bool &ore, float &val);
template <>
__device__ __forceinline__ void relax_ore_value<float>(const float *g, const RelaxRows &, int32_t b, int32_t S, int s,
                                                       float m, const RelaxEcon &E, bool &ore, float &val) {
    const float gv = __ldg(g + (size_t)b * S + s);
    ore = relax_ore(gv, E);
    const float mc = m * E.mcf;
    val = ore ? m * ((gv * E.pf) * E.rf - E.pcf) - mc : -mc;
}
template <>
__device__ __forceinline__ void relax_ore_value<double>(const double *, const RelaxRows &Rw, int32_t b, int32_t, int s,
                                                        float, const RelaxEcon &, bool &ore, float &val) {
    const float *row = Rw.val + (size_t)b * Rw.R;
    val = __ldg(row + s);
    ore = (__ldg(reinterpret_cast<const uint32_t *>(row + Rw.ore_off) + (s >> 5)) >> (s & 31)) & 1u;
}

// Forward contraction, staged: CTA (r, z) owns the contiguous range r of the
// blocks and scenario tile z (up to kFwdSW scenarios) for one tile of TT
// periods starting at t0 (TT a multiple of 4: the staged x rows are read four
// periods at a time).  Tiles of kFwdBT blocks -- the grade slices (caller
// grades) or value slices and ore words (model rows), the x rows and the
// masses -- are copied into shared memory by cp.async, up to kFwdStages - 1
// tiles ahead of the one being summed, so every grade is read from memory
// once and many copies are in flight.  The CTA's kFwdGroups thread groups
// split each tile's blocks (group k takes blocks k, k + kFwdGroups, ...);
// thread s of a group sums x[b][t] m_b ore[b][s] and x[b][t] v[b][s] in FP32
// registers, the groups' sums are added in group order through shared memory
// and the CTA writes one partial of O and V; the partials are added in FP64 in
// range order afterwards (deterministic).
constexpr int kFwdBT = 24;      // blocks per staged tile (three stages stay under 48 KB of static shared memory)
constexpr int kFwdStages = 3;   // staged tiles (two in flight while one is summed)
constexpr int kFwdSW = 128;     // scenarios per CTA (at most)
constexpr int kFwdGroups = 2;   // thread groups splitting a tile's blocks
#ifndef MM_RELAX_CTAS_PER_SM
#define MM_RELAX_CTAS_PER_SM 2      // forward CTAs per SM (each writes one partial)
#endif

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// Two FP32 values in one 64-bit register pair and the paired FMA of the
// sm_100 family (each lane rounded exactly like the scalar fmaf).
__device__ __forceinline__ uint64_t rx_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void rx_unpack(uint64_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t rx_fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <typename G, int TT>
__global__ void __launch_bounds__(kFwdSW * kFwdGroups) k_relax_fwd(const float *__restrict__ x, const G *__restrict__ g,
                                                      RelaxRows Rw, const uint32_t *__restrict__ mass, int32_t B,
                                                      int32_t S, int32_t T, int32_t t0, RelaxEcon E, int32_t vec,
                                                      int32_t xvec, float *__restrict__ part_o,
                                                      float *__restrict__ part_v) {
    constexpr bool ROWS = sizeof(G) == sizeof(double);          // model rows: values, then ore words
    constexpr int RW = kFwdSW + (ROWS ? 4 : 0);                  // staged floats per block
    __shared__ __align__(16) float s_g[kFwdStages][kFwdBT][RW];
    __shared__ __align__(16) float s_x[kFwdStages][kFwdBT][TT];
    __shared__ uint32_t s_m[kFwdStages][kFwdBT];
    const int r = blockIdx.x, nr = gridDim.x;
    const int b_lo = (int)((int64_t)r * B / nr), b_hi = (int)((int64_t)(r + 1) * B / nr);
    const int s0 = blockIdx.z * kFwdSW, sw = min(kFwdSW, S - s0);
    const int nt = min(TT, T - t0);
    const int ntiles = (b_hi - b_lo + kFwdBT - 1) / kFwdBT;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    // the groups are packed: group k is threads [k gw, (k + 1) gw), gw the
    // widest scenario tile, so that few lanes idle when S is not a multiple of
    // 32 (threads from kFwdGroups gw on only copy)
    const int gw = min(S, kFwdSW);
    const int grp = tid / gw, lt = tid - grp * gw;   // group, scenario lane
    auto issue = [&](int k) {
        const int st = k % kFwdStages, bb0 = b_lo + k * kFwdBT, nb = min(kFwdBT, b_hi - bb0);
        // one warp per block row, one lane per 16 (or 4) bytes: no divisions
        if (ROWS) {
            // value slice [s0, s0 + sw) rounded up to 16 bytes (the row's zero padding
            // runs to a multiple of 4 floats) and the slice's ore words (one 16-byte copy)
            const int nv4 = (sw + 3) / 4, per = nv4 + 1;
            for (int j = warp; j < nb; j += nwarps) {
                const float *row = Rw.val + (size_t)(bb0 + j) * Rw.R;
                for (int q = lane; q < per; q += 32) {
                    if (q < nv4) cp_async16(&s_g[st][j][4 * q], row + s0 + 4 * q);
                    else cp_async16(&s_g[st][j][kFwdSW], row + Rw.ore_off + s0 / 32);
                }
            }
        } else if (vec) {
            const int nv4 = sw / 4;  // S % 4 == 0
            for (int j = warp; j < nb; j += nwarps) {
                const float *row = reinterpret_cast<const float *>(g) + (size_t)(bb0 + j) * S + s0;
                for (int q = lane; q < nv4; q += 32) cp_async16(&s_g[st][j][4 * q], row + 4 * q);
            }
        } else {
            for (int j = warp; j < nb; j += nwarps) {
                const float *row = reinterpret_cast<const float *>(g) + (size_t)(bb0 + j) * S + s0;
                for (int q = lane; q < sw; q += 32) cp_async4(&s_g[st][j][q], row + q);
            }
        }
        if (xvec) {
            // T % 4 == 0 (so t0, nt and every row start are multiples of 4 floats):
            // the tile's x rows in 16-byte pieces, nt / 4 per block
            const int n4 = nt >> 2;
            for (int i = tid; i < nb * n4; i += nth) {
                const int j = i / n4, q = i - j * n4;
                cp_async16(&s_x[st][j][4 * q], x + (size_t)(bb0 + j) * T + t0 + 4 * q);
            }
        } else {
            for (int j = warp; j < nb; j += nwarps)
                for (int q = lane; q < nt; q += 32) cp_async4(&s_x[st][j][q], x + (size_t)(bb0 + j) * T + t0 + q);
        }
        for (int j = tid; j < nb; j += nth) cp_async4(&s_m[st][j], mass + bb0 + j);
    };
    // periods t0 + nt .. t0 + TT - 1 of the x tiles stay zero
    if (nt < TT)
        for (int i = tid; i < kFwdStages * kFwdBT * TT; i += nth) (&s_x[0][0][0])[i] = 0.0f;
    __syncthreads();
    // always kFwdStages - 1 groups (empty ones past the last tile), so that the
    // wait below counts the same groups for every range length
    for (int k = 0; k < kFwdStages - 1; k++) {
        if (k < ntiles) issue(k);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const bool live = grp < kFwdGroups && lt < sw;
    const int s = s0 + lt;
    uint64_t o2[TT / 2], v2[TT / 2];  // period pairs (2q, 2q + 1)
#pragma unroll
    for (int j = 0; j < TT / 2; j++) o2[j] = v2[j] = 0ull;
    for (int k = 0; k < ntiles; k++) {
        if (k + kFwdStages - 1 < ntiles) issue(k + kFwdStages - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group %0;" ::"n"(kFwdStages - 1) : "memory");  // tile k has landed
        __syncthreads();
        const int st = k % kFwdStages, nb = min(kFwdBT, b_hi - (b_lo + k * kFwdBT));
        if (live) {
            // the next block's grade (or value and ore word) and mass are read
            // from shared memory before the current block's products
            int j = grp;
            float g_n = 0.0f;
            uint32_t w_n = 0u, m_n = 0u;
            if (j < nb) {
                g_n = s_g[st][j][lt];
                if (ROWS) w_n = __float_as_uint(s_g[st][j][kFwdSW + (lt >> 5)]);
                m_n = s_m[st][j];
            }
#pragma unroll 4
            for (; j < nb; j += kFwdGroups) {
                const float gv = g_n, m = (float)m_n;
                const uint32_t ow = w_n;
                const int jn = j + kFwdGroups;
                if (jn < nb) {
                    g_n = s_g[st][jn][lt];
                    if (ROWS) w_n = __float_as_uint(s_g[st][jn][kFwdSW + (lt >> 5)]);
                    m_n = s_m[st][jn];
                }
                float val;
                bool ore;
                if (ROWS) {
                    val = gv;
                    ore = (ow >> (lt & 31)) & 1u;
                } else {
                    ore = relax_ore(gv, E);
                    const float mc = m * E.mcf;
                    val = ore ? m * ((gv * E.pf) * E.rf - E.pcf) - mc : -mc;
                }
                const float mo = ore ? m : 0.0f;
                const uint64_t mo2 = rx_pack(mo, mo), val2 = rx_pack(val, val);
                const float4 *xr = reinterpret_cast<const float4 *>(s_x[st][j]);
#pragma unroll
                for (int q = 0; q < TT / 4; q++) {
                    const float4 x4 = xr[q];
                    const uint64_t xa = rx_pack(x4.x, x4.y), xb = rx_pack(x4.z, x4.w);
                    o2[2 * q] = rx_fma2(xa, mo2, o2[2 * q]);
                    o2[2 * q + 1] = rx_fma2(xb, mo2, o2[2 * q + 1]);
                    v2[2 * q] = rx_fma2(xa, val2, v2[2 * q]);
                    v2[2 * q + 1] = rx_fma2(xb, val2, v2[2 * q + 1]);
                }
            }
        }
        __syncthreads();  // stage k % kFwdStages is refilled next
    }
    float o[TT], v[TT];
#pragma unroll
    for (int j = 0; j < TT / 2; j++) {
        rx_unpack(o2[j], o[2 * j], o[2 * j + 1]);
        rx_unpack(v2[j], v[2 * j], v[2 * j + 1]);
    }
    // groups 1.. hand their sums to group 0 through the (now idle) grade
    // stages, which group 0 adds in group order
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    float *red = &s_g[0][0][0];  // [kFwdGroups - 1][2][TT][kFwdSW]
    static_assert((kFwdGroups - 1) * 2 * TT * kFwdSW <= kFwdStages * kFwdBT * RW, "combine space");
    if (grp > 0 && live) {
#pragma unroll
        for (int j = 0; j < TT; j++) {
            red[(((size_t)(grp - 1) * 2) * TT + j) * kFwdSW + lt] = o[j];
            red[(((size_t)(grp - 1) * 2 + 1) * TT + j) * kFwdSW + lt] = v[j];
        }
    }
    __syncthreads();
    if (grp == 0 && live) {
#pragma unroll
        for (int j = 0; j < TT; j++) {
            float a = o[j], c = v[j];
#pragma unroll
            for (int k = 1; k < kFwdGroups; k++) {
                a += red[(((size_t)(k - 1) * 2) * TT + j) * kFwdSW + lt];
                c += red[(((size_t)(k - 1) * 2 + 1) * TT + j) * kFwdSW + lt];
            }
            if (j < nt) {
                part_o[((size_t)r * T + t0 + j) * S + s] = a;
                part_v[((size_t)r * T + t0 + j) * S + s] = c;
            }
        }
    }
}

template <typename G>
static mm_status relax_fwd_launch(const float *x, const G *g, RelaxRows Rw, const uint32_t *mass, int32_t B, int32_t S,
                                  int32_t T, RelaxEcon E, float *part_o, float *part_v, int nr, cudaStream_t st) {
    const int zs = (S + kFwdSW - 1) / kFwdSW;
    const int threads = (kFwdGroups * std::min(S, kFwdSW) + 31) / 32 * 32;
    const int vec = (S % 4 == 0 && ((uintptr_t)g & 15u) == 0) ? 1 : 0;
    const int xvec = (T % 4 == 0 && ((uintptr_t)x & 15u) == 0) ? 1 : 0;  // period tiles start at multiples of 4
    static_assert(kRelaxTile % 4 == 0, "period tiles must start at multiples of 4 floats");
    for (int tb = 0; tb < T; tb += kRelaxTile) {
        const int tt = (std::min(kRelaxTile, T - tb) + 3) / 4 * 4;
        const dim3 grid(nr, 1, zs);
        switch (tt) {
            case 4: k_relax_fwd<G, 4><<<grid, threads, 0, st>>>(x, g, Rw, mass, B, S, T, tb, E, vec, xvec, part_o, part_v); break;
            case 8: k_relax_fwd<G, 8><<<grid, threads, 0, st>>>(x, g, Rw, mass, B, S, T, tb, E, vec, xvec, part_o, part_v); break;
            case 12: k_relax_fwd<G, 12><<<grid, threads, 0, st>>>(x, g, Rw, mass, B, S, T, tb, E, vec, xvec, part_o, part_v); break;
            case 16: k_relax_fwd<G, 16><<<grid, threads, 0, st>>>(x, g, Rw, mass, B, S, T, tb, E, vec, xvec, part_o, part_v); break;
            case 20: k_relax_fwd<G, 20><<<grid, threads, 0, st>>>(x, g, Rw, mass, B, S, T, tb, E, vec, xvec, part_o, part_v); break;
            default: k_relax_fwd<G, 24><<<grid, threads, 0, st>>>(x, g, Rw, mass, B, S, T, tb, E, vec, xvec, part_o, part_v); break;
        }
        mm_status r = check_launch("k_relax_fwd");
        if (r != MM_OK) return r;
    }
    return MM_OK;
}

// softplus and its derivative of beta z, the argument formed in FP64 and the
// transcendental part in FP32 (relative error ~1e-7 of a term far below the
// NPV and gradient tolerances).
__device__ __forceinline__ double relax_softplus(double z, const RelaxEcon &E) {
    const double bz = E.beta * z;
    const float abz = (float)fabs(bz);
    return (fmax(bz, 0.0) + (double)log1pf(expf(-abz))) * E.inv_beta;
}
__device__ __forceinline__ double relax_sigmoid(double z, double beta) {
    return (double)(1.0f / (1.0f + expf((float)(-beta * z))));
}

// FP64 sum over the threads of one CTA (valid in every thread): xor trees
// inside each warp and then over the warp sums (a fixed order, ten dependent
// additions rather than one per warp).
__device__ double relax_block_sum(double x, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    const double r = red[32];
    __syncthreads();
    return r;
}

// (sum of x, sum of x^2) over the threads of one CTA in FP64, the two chains
// side by side (valid in every thread); the same fixed trees as
// relax_block_sum.
__device__ double2 relax_block_sum2(double x, double y, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, off);
        y += __shfl_xor_sync(0xffffffffu, y, off);
    }
    if (lane == 0) {
        red[warp] = x;
        red[32 + warp] = y;
    }
    __syncthreads();
    if (warp == 0) {
        double a = lane < nw ? red[lane] : 0.0, b = lane < nw ? red[32 + lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            b += __shfl_xor_sync(0xffffffffu, b, off);
        }
        if (lane == 0) {
            red[64] = a;
            red[65] = b;
        }
    }
    __syncthreads();
    const double2 r = make_double2(red[64], red[65]);
    __syncthreads();
    return r;
}

// Neumaier-compensated FP32 accumulation (s, c) += x, and the merge of two
// compensated sums.
__device__ __forceinline__ void relax_neumaier(float &s, float &c, float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}
__device__ __forceinline__ void relax_merge(float &s, float &c, float s2, float c2) {
    relax_neumaier(s, c, s2);
    c += c2;
}

// End of the forward pass, one launch:
//   1. O[t][s] and V[t][s] from the range partials: a CTA of 32 warps per 32
//      consecutive (t, s) (coalesced), warp w adding ranges w, w + 32, ... by
//      compensated FP32 sums, the 32 warp sums merged by a fixed pairwise
//      tree (deterministic; the error is about one FP32 rounding of the
//      total, with no FP64 work on the long sums);
//   2. the FP64 checkpoint O[t][s] and term[t][s] = d_t (V - P_t(O));
//   3. the last CTA to finish (acquire-release ticket) forms
//      NPV_s = sum_t term[t][s] in period order, the mean and population std
//      over scenarios and J, and resets the ticket.
__global__ void __launch_bounds__(1024) k_relax_finish(const float *__restrict__ part_o,
                                                       const float *__restrict__ part_v, int32_t nr, int32_t S,
                                                       int32_t T, const double *__restrict__ disc,
                                                       const uint64_t *__restrict__ target, RelaxEcon E,
                                                       double *__restrict__ o_out, double *term, uint32_t *tick,
                                                       double *__restrict__ npv, double *__restrict__ J) {
    __shared__ float s_sum[2][32][32], s_cmp[2][32][32];  // [O / V][warp][lane]
    __shared__ double red[66];
    __shared__ int s_last;
    const int TS = T * S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    float so = 0.0f, co = 0.0f, sv = 0.0f, cv = 0.0f;
    if (i < TS) {
        // eight ranges' partials loaded before any is added
        for (int c0 = warp; c0 < nr; c0 += 8 * 32) {
            float a[8], b[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int c = c0 + 32 * u;
                a[u] = c < nr ? __ldg(part_o + (size_t)c * TS + i) : 0.0f;
                b[u] = c < nr ? __ldg(part_v + (size_t)c * TS + i) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                relax_neumaier(so, co, a[u]);
                relax_neumaier(sv, cv, b[u]);
            }
        }
    }
    s_sum[0][warp][lane] = so; s_cmp[0][warp][lane] = co;
    s_sum[1][warp][lane] = sv; s_cmp[1][warp][lane] = cv;
    __syncthreads();
#pragma unroll
    for (int h = 16; h > 0; h >>= 1) {
        if (warp < h) {
#pragma unroll
            for (int q = 0; q < 2; q++) {
                float a = s_sum[q][warp][lane], b = s_cmp[q][warp][lane];
                relax_merge(a, b, s_sum[q][warp + h][lane], s_cmp[q][warp + h][lane]);
                s_sum[q][warp][lane] = a;
                s_cmp[q][warp][lane] = b;
            }
        }
        __syncthreads();
    }
    if (warp == 0 && i < TS) {
        const double O = (double)s_sum[0][0][lane] + (double)s_cmp[0][0][lane];
        const double V = (double)s_sum[1][0][lane] + (double)s_cmp[1][0][lane];
        o_out[i] = O;
        const int t = i / S;
        const double Q = (double)target[t];
        const double pen = E.a * E.m_ref * relax_softplus((Q - O) * E.inv_mref, E) +
                           E.e * E.m_ref * relax_softplus((O - Q) * E.inv_mref, E);
        term[i] = disc[t] * (V - pen);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t old;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(tick) : "memory");
        s_last = old == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    const int s = threadIdx.x;
    double acc = 0.0;
    if (s < S) {
        // periods in batches of eight, loaded together and added by a fixed
        // pairwise tree, the batch sums in period order (short FP64 chains)
        for (int t0 = 0; t0 < T; t0 += 8) {
            double q[8];
#pragma unroll
            for (int u = 0; u < 8; u++) q[u] = t0 + u < T ? __ldcg(term + (size_t)(t0 + u) * S + s) : 0.0;
            acc += ((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + (q[6] + q[7]));
        }
        npv[s] = acc;
    }
    // mean and population variance in one pass of (sum, sum of squares)
    const double2 sums = relax_block_sum2(s < S ? acc : 0.0, s < S ? acc * acc : 0.0, red);
    const double mean = sums.x * E.inv_S;
    const double var = fmax(sums.y * E.inv_S - mean * mean, 0.0);
    if (s == 0) {
        J[0] = mean - E.lambda * sqrt(var);
        *tick = 0u;
    }
}

// Adjoint coefficients: w_s = gJ (1/S - lambda (NPV_s - mean) / (S std))
// (the std term dropped where std = 0) and c[t][s] = w_s P_t'(O[t][s]), one
// thread per (t, s) over many CTAs; every CTA forms mean and std itself.
__global__ void __launch_bounds__(256) k_relax_coef(const double *__restrict__ npv, const double *__restrict__ o,
                                                    const uint64_t *__restrict__ target, const double *__restrict__ gJ,
                                                    int32_t S, int32_t T, int32_t Sp, RelaxEcon E,
                                                    float *__restrict__ w_out, float *__restrict__ c_out) {
    __shared__ double red[33];
    double part = 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) part += npv[s];
    const double mean = relax_block_sum(part, red) * E.inv_S;
    double pv = 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double d = npv[s] - mean;
        pv += d * d;
    }
    const double sd = sqrt(relax_block_sum(pv, red) * E.inv_S);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T * S) return;
    const int t = i / S, s = i - t * S;
    const double g = gJ[0];
    double w = g * E.inv_S;
    if (sd > 0.0) w -= g * E.lambda * (npv[s] - mean) * E.inv_S / sd;
    if (t == 0) w_out[s] = (float)w;
    const double O = o[i], Q = (double)target[t];
    const double dp = -E.a * relax_sigmoid((Q - O) * E.inv_mref, E.beta) + E.e * relax_sigmoid((O - Q) * E.inv_mref, E.beta);
    c_out[(size_t)t * Sp + s] = (float)(w * dp);
}

// dJ/dx and dJ/dg, one warp per block.  Shared memory: w[S], c[T][Sp] (Sp odd:
// lane t reads row t without bank conflicts), d[T], the warp's ore bits.
// Tiled adjoint (the fast path): a tile of kAdjBT blocks at a time, one per
// lane.  The tile's grades (or values and ore words), x rows and masses go to
// shared memory by asynchronous 4-byte copies, all in flight at once (reads
// coalesced along each row); warp w takes scenarios w, w + 8, ... and
// keeps, per block (lane), u = sum_s w_s v[b][s] and A[t] = sum_s c[t][s]
// ore[b][s] for the period tile t0 .. t0 + TT - 1 in registers (period pairs,
// paired FMAs; c is held transposed, [s][TT]); the eight warps' partial sums
// are added in warp order; then
//   dJ/dx[b][t] = d_t (u_b - m_b A[t]),
//   dJ/dg[b][s] = w_s ore[b][s] m_b price recovery sum_t d_t x[b][t]  (t0 == 0),
// both written coalesced.  Persistent: CTA i takes tiles i, i + grid, ...
constexpr int kAdjBT = 32;
constexpr int kAdjWarps = 8;

struct AdjLayout {
    int Sg, Wo, TT4;  // odd grade row stride, odd ore-word row stride, padded period tile
    size_t c, w, d, D, acc, g, ow, x, m, floats;
};
__host__ __device__ inline AdjLayout adj_layout(int S, int T, int TT, bool rows) {
    AdjLayout L;
    L.Sg = S | 1;
    L.Wo = rows ? (((S + 31) / 32) | 1) : 0;
    L.TT4 = TT;
    L.c = 0;                                        // [S][TT]
    L.w = L.c + (size_t)S * TT;                     // [S]
    L.d = L.w + S;                                  // [T]
    L.D = L.d + T;                                  // [kAdjBT]
    L.acc = L.D + kAdjBT;                           // [kAdjWarps][TT + 1][kAdjBT]
    L.g = L.acc + (size_t)kAdjWarps * (TT + 1) * kAdjBT;  // [kAdjBT][Sg]
    L.ow = L.g + (size_t)kAdjBT * L.Sg;             // [kAdjBT][Wo] (u32)
    L.x = L.ow + (size_t)kAdjBT * L.Wo;             // [kAdjBT * T]
    L.m = L.x + (size_t)kAdjBT * T;                 // [kAdjBT] (u32 masses)
    L.floats = L.m + kAdjBT;
    return L;
}

template <typename G, int TT>
__global__ void __launch_bounds__(32 * kAdjWarps) k_relax_adj_tiled(const float *__restrict__ x,
                                                                     const G *__restrict__ g, RelaxRows Rw,
                                                                     const uint32_t *__restrict__ mass,
                                                                     const float *__restrict__ w,
                                                                     const float *__restrict__ c,
                                                                     const double *__restrict__ disc, int32_t B,
                                                                     int32_t S, int32_t T, int32_t Sp, int32_t t0,
                                                                     RelaxEcon E, float *__restrict__ gx,
                                                                     float *__restrict__ gg) {
    constexpr bool ROWS = sizeof(G) == sizeof(double);
    extern __shared__ __align__(16) float sm[];
    const AdjLayout L = adj_layout(S, T, TT, ROWS);
    float *s_c = sm + L.c, *s_w = sm + L.w, *s_d = sm + L.d, *s_D = sm + L.D;
    float *s_acc = sm + L.acc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nth = blockDim.x;
    const int nt = min(TT, T - t0);
    // per CTA: c transposed to [s][TT] (zero past the period tile), w, d
    for (int q = nt + warp; q < TT; q += kAdjWarps)
        for (int sc = lane; sc < S; sc += 32) s_c[(size_t)sc * TT + q] = 0.0f;
    for (int q = warp; q < nt; q += kAdjWarps)
        for (int sc = lane; sc < S; sc += 32) cp_async4(&s_c[(size_t)sc * TT + q], c + (size_t)(t0 + q) * Sp + sc);
    for (int i = tid; i < S; i += nth) cp_async4(&s_w[i], w + i);
    for (int i = tid; i < T; i += nth) s_d[i] = (float)disc[i];
    const float prf = E.pf * E.rf;
    const int ntile = (B + kAdjBT - 1) / kAdjBT;
    float *s_g = sm + L.g, *s_x = sm + L.x;
    uint32_t *s_ow = reinterpret_cast<uint32_t *>(sm + L.ow), *s_m = reinterpret_cast<uint32_t *>(sm + L.m);
    for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int b0 = tile * kAdjBT, nb = min(kAdjBT, B - b0);
        // stage the tile: a warp per block row, lanes along the row, every
        // copy in flight at once (the first tile's join those of c and w)
        for (int j = warp; j < nb; j += kAdjWarps) {
            if (ROWS) {
                const float *row = Rw.val + (size_t)(b0 + j) * Rw.R;
                for (int sc = lane; sc < S; sc += 32) cp_async4(&s_g[j * L.Sg + sc], row + sc);
                for (int k = lane; k < (S + 31) / 32; k += 32) cp_async4(&s_ow[j * L.Wo + k], row + Rw.ore_off + k);
            } else {
                const float *row = reinterpret_cast<const float *>(g) + (size_t)(b0 + j) * S;
                for (int sc = lane; sc < S; sc += 32) cp_async4(&s_g[j * L.Sg + sc], row + sc);
            }
        }
        for (int i = tid; i < nb * T; i += nth) cp_async4(&s_x[i], x + (size_t)b0 * T + i);
        for (int j = tid; j < nb; j += nth) cp_async4(&s_m[j], mass + b0 + j);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        const bool have = lane < nb;
        const float m = have ? (float)s_m[lane] : 0.0f;
        if (warp == 0 && have) {
            float D = 0.0f;
            for (int t = 0; t < T; t++) D = fmaf(s_d[t], s_x[lane * T + t], D);
            s_D[lane] = D;
        }
        // per-warp sums over scenarios warp, warp + 8, ... for block `lane`
        uint64_t a2[TT / 2];
#pragma unroll
        for (int q = 0; q < TT / 2; q++) a2[q] = 0ull;
        float u = 0.0f;
        if (have) {
            const float *grow = s_g + lane * L.Sg;
            for (int sc = warp; sc < S; sc += kAdjWarps) {
                const float gv = grow[sc];
                bool ore;
                float val;
                if (ROWS) {
                    val = gv;
                    ore = (s_ow[lane * L.Wo + (sc >> 5)] >> (sc & 31)) & 1u;
                } else {
                    ore = relax_ore(gv, E);
                    const float mc = m * E.mcf;
                    val = ore ? m * ((gv * E.pf) * E.rf - E.pcf) - mc : -mc;
                }
                u = fmaf(s_w[sc], val, u);
                const float of = ore ? 1.0f : 0.0f;
                const uint64_t of2 = rx_pack(of, of);
                const float4 *cr = reinterpret_cast<const float4 *>(s_c + (size_t)sc * TT);
#pragma unroll
                for (int q = 0; q < TT / 4; q++) {
                    const float4 c4 = cr[q];
                    a2[2 * q] = rx_fma2(rx_pack(c4.x, c4.y), of2, a2[2 * q]);
                    a2[2 * q + 1] = rx_fma2(rx_pack(c4.z, c4.w), of2, a2[2 * q + 1]);
                }
            }
        }
        // partial sums to shared memory: [warp][TT + 1][lane] (row TT = u)
        float *my = s_acc + (size_t)warp * (TT + 1) * kAdjBT;
#pragma unroll
        for (int q = 0; q < TT / 2; q++) {
            float lo, hi;
            rx_unpack(a2[q], lo, hi);
            my[(2 * q) * kAdjBT + lane] = lo;
            my[(2 * q + 1) * kAdjBT + lane] = hi;
        }
        my[TT * kAdjBT + lane] = u;
        __syncthreads();
        // warp-order sums into warp 0's slot
        for (int i = tid; i < (TT + 1) * kAdjBT; i += nth) {
            float a = s_acc[i];
#pragma unroll
            for (int k = 1; k < kAdjWarps; k++) a += s_acc[(size_t)k * (TT + 1) * kAdjBT + i];
            s_acc[i] = a;
        }
        __syncthreads();
        // dJ/dx of the period tile and dJ/dg (once, with the first period
        // tile): a warp per block row, lanes along the row
        for (int j = warp; j < nb; j += kAdjWarps) {
            const float mj = (float)s_m[j];
            for (int q = lane; q < nt; q += 32)
                gx[(size_t)(b0 + j) * T + t0 + q] = s_d[t0 + q] * (s_acc[TT * kAdjBT + j] - mj * s_acc[q * kAdjBT + j]);
            if (gg && t0 == 0) {
                const float f = mj * prf * s_D[j];
                for (int sc = lane; sc < S; sc += 32) {
                    bool ore;
                    if (ROWS) ore = (s_ow[j * L.Wo + (sc >> 5)] >> (sc & 31)) & 1u;
                    else ore = relax_ore(s_g[j * L.Sg + sc], E);
                    gg[(size_t)(b0 + j) * S + sc] = ore ? s_w[sc] * f : 0.0f;
                }
            }
        }
        __syncthreads();  // the tile's shared data and sums are read no more before they are refilled
    }
}

template <typename G>
__global__ void __launch_bounds__(256) k_relax_adjoint(const float *__restrict__ x, const G *__restrict__ g,
                                                       RelaxRows Rw, const uint32_t *__restrict__ mass,
                                                       const float *__restrict__ w,
                                                       const float *__restrict__ c, const double *__restrict__ disc,
                                                       int32_t B, int32_t S, int32_t T, int32_t Sp, RelaxEcon E,
                                                       float *__restrict__ gx, float *__restrict__ gg) {
    extern __shared__ __align__(16) float s_relax[];
    const int W = (S + 31) / 32;
    float *s_w = s_relax;                              // [S]
    float *s_c = s_w + S;                              // [T][Sp]
    float *s_d = s_c + (size_t)T * Sp;                 // [T]
    float *s_call = s_d + T;                           // [T] sum_s c[t][s]
    uint32_t *s_ore = reinterpret_cast<uint32_t *>(s_call + T);  // [warps][W]
    for (int i = threadIdx.x; i < S; i += blockDim.x) s_w[i] = w[i];
    for (int i = threadIdx.x; i < T * Sp; i += blockDim.x) s_c[i] = c[i];
    for (int i = threadIdx.x; i < T; i += blockDim.x) s_d[i] = (float)disc[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = warp; t < T; t += (int)(blockDim.x >> 5)) {
        float a = 0.0f;
        for (int s = lane; s < S; s += 32) a += s_c[(size_t)t * Sp + s];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) s_call[t] = a;
    }
    __syncthreads();
    uint32_t *ore_w = s_ore + (size_t)warp * W;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const float prf = E.pf * E.rf;
    for (int b = blockIdx.x * (blockDim.x >> 5) + warp; b < B; b += nwarps) {
        const float m = (float)mass[b];
        // u = sum_s w_s v[b][s]; ore bits of the block and their count
        float u = 0.0f;
        int nore = 0;
        for (int s0 = 0; s0 < S; s0 += 32) {
            const int s = s0 + lane;
            bool ore = false;
            if (s < S) {
                float val;
                relax_ore_value<G>(g, Rw, b, S, s, m, E, ore, val);
                u = fmaf(s_w[s], val, u);
            }
            const uint32_t bits = __ballot_sync(0xffffffffu, ore);
            nore += __popc(bits);
            if (lane == 0) ore_w[s0 >> 5] = bits;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) u += __shfl_xor_sync(0xffffffffu, u, off);
        // D = sum_t d_t x[b][t]
        float D = 0.0f;
        for (int t = lane; t < T; t += 32) D = fmaf(s_d[t], x[(size_t)b * T + t], D);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) D += __shfl_xor_sync(0xffffffffu, D, off);
        __syncwarp();
        // dJ/dg
        if (gg) {
            const float f = m * prf * D;
            for (int s = lane; s < S; s += 32) {
                const bool ore = (ore_w[s >> 5] >> (s & 31)) & 1u;
                gg[(size_t)b * S + s] = ore ? s_w[s] * f : 0.0f;
            }
        }
        // dJ/dx: lane t forms sum_s c[t][s] ore[b][s] over the ore scenarios,
        // or as the row total minus the waste scenarios when those are fewer
        const bool cmpl = 2 * nore > S;
        for (int t = lane; t < T; t += 32) {
            const float *crow = s_c + (size_t)t * Sp;
            float acc = 0.0f;
            for (int k = 0; k < W; k++) {
                uint32_t bits = cmpl ? ~ore_w[k] : ore_w[k];
                if (k == W - 1 && (S & 31)) bits &= (1u << (S & 31)) - 1u;
                while (bits) {
                    const int j = __ffs(bits) - 1;
                    bits &= bits - 1;
                    acc += crow[k * 32 + j];
                }
            }
            gx[(size_t)b * T + t] = s_d[t] * (u - m * (cmpl ? s_call[t] - acc : acc));
        }
        __syncwarp();
    }
}

static mm_status relax_scratch(mm_model *m, size_t floats) {
    if (m->relax_scratch_floats >= floats) return MM_OK;
    cudaFree(m->relax_scratch);
    m->relax_scratch = nullptr;
    m->relax_scratch_floats = 0;
    MM_CUDA_TRY(cudaMalloc(&m->relax_scratch, floats * sizeof(float)), "allocate relaxed-objective scratch");
    m->relax_scratch_floats = floats;
    return MM_OK;
}

// The FP64 ore test of a float grade, exactly as the kernels would form it.
static bool host_ore(float g, double p, double r, double pc) {
    volatile double gp = (double)g * p;  // each product rounded to double, in this order
    volatile double gpr = gp * r;
    return gpr > pc;
}

static RelaxEcon relax_econ(const mm_model *m, double beta, double m_ref) {
    RelaxEcon E;
    E.p = m->price; E.r = m->recovery; E.pc = m->proc_cost;
    E.pf = (float)m->price; E.rf = (float)m->recovery; E.pcf = (float)m->proc_cost; E.mcf = (float)m->mining_cost;
    E.a = m->shortfall_pen; E.e = m->excess_pen; E.lambda = m->lambda; E.beta = beta; E.m_ref = m_ref;
    E.inv_beta = 1.0 / beta; E.inv_mref = 1.0 / m_ref; E.inv_S = 1.0 / m->S;
    // (g p) r > pc is non-decreasing in g >= 0 when p, r > 0, and false for
    // g < 0 when pc >= 0: the smallest non-negative float with the test true
    // (binary search over the ordered bit patterns of 0 .. +inf) is g_t
    E.use_thr = m->price > 0.0 && m->recovery > 0.0 && m->proc_cost >= 0.0;
    E.g_thr = INFINITY;
    if (E.use_thr) {
        uint32_t lo = 0u, hi = 0x7f800000u;  // bit patterns of 0.0f and +inf
        auto f = [&](uint32_t bits) {
            float g;
            std::memcpy(&g, &bits, sizeof g);
            return host_ore(g, m->price, m->recovery, m->proc_cost);
        };
        if (f(lo)) {
            E.g_thr = 0.0f;
        } else if (f(hi)) {
            while (hi - lo > 1u) {
                const uint32_t mid = lo + (hi - lo) / 2u;
                if (f(mid)) hi = mid;
                else lo = mid;
            }
            std::memcpy(&E.g_thr, &hi, sizeof hi);
        }
    }
    return E;
}

static mm_status relax_check(mm_model *m, const float *x, double beta, double m_ref) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (m->sig) return set_error(MM_ERR_INVALID_ARG, "the relaxed objective does not take uncertainty weights");
    if (!x) return set_error(MM_ERR_INVALID_ARG, "NULL x");
    if (!(beta > 0.0) || !(m_ref > 0.0) || !std::isfinite(beta) || !std::isfinite(m_ref))
        return set_error(MM_ERR_INVALID_ARG, "beta and m_ref must be positive and finite");
    return MM_OK;
}

// First-order prior of candidate moves from dJ/dx at the one-hot schedule:
// one thread per move, the periods from the packed schedule words.
__global__ void __launch_bounds__(256) k_relax_prior(const float *__restrict__ gx, const int2 *__restrict__ moves,
                                                     int64_t n, int32_t B, int32_t T,
                                                     const uint32_t *__restrict__ blk, uint32_t *status,
                                                     float *__restrict__ prior) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int2 mv = __ldg(moves + i);
        const bool swap = mv.y >= 0;
        const int64_t tn = -(int64_t)mv.y - 1;
        const bool valid = mv.x >= 0 && mv.x < B && (swap ? mv.y < B : (tn >= 0 && tn <= (int64_t)T));
        if (!valid) {
            prior[i] = -INFINITY;
            atomicOr(status, kStBadMove);
            continue;
        }
        auto g = [&](int32_t b, uint32_t t) { return t < (uint32_t)T ? __ldg(gx + (size_t)b * T + t) : 0.0f; };
        const uint32_t t1 = blk_period(__ldg(blk + mv.x));
        if (swap) {
            const uint32_t t2 = blk_period(__ldg(blk + mv.y));
            prior[i] = (g(mv.x, t2) - g(mv.x, t1)) + (g(mv.y, t1) - g(mv.y, t2));
        } else {
            prior[i] = g(mv.x, (uint32_t)tn) - g(mv.x, t1);
        }
    }
}

}  // namespace mm

using namespace mm;

extern "C" {

mm_status mm_relaxed_move_prior(mm_model *m, const float *gx_dev, const mm_move *moves, int64_t n, float *prior) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    if (n < 0) return set_error(MM_ERR_INVALID_ARG, "negative move count");
    if (n == 0) return MM_OK;
    if (!gx_dev || !moves || !prior) return set_error(MM_ERR_INVALID_ARG, "NULL gradient, move or output pointer");
    if (((uintptr_t)moves & 7u) != 0) return set_error(MM_ERR_INVALID_ARG, "moves must be 8-byte aligned");
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)m->num_sms * 8) blocks = (int64_t)m->num_sms * 8;
    k_relax_prior<<<(unsigned)blocks, 256, 0, m->stream>>>(gx_dev, reinterpret_cast<const int2 *>(moves), n, m->B,
                                                            m->T, m->blk, m->status, prior);
    return check_launch("k_relax_prior");
}

mm_status mm_relaxed_forward(mm_model *m, const float *x_dev, const float *g_dev, double beta, double m_ref,
                             double *J_dev, double *npv_dev, double *ore_t_dev) {
    mm_status st = relax_check(m, x_dev, beta, m_ref);
    if (st != MM_OK) return st;
    if (!J_dev || !npv_dev || !ore_t_dev) return set_error(MM_ERR_INVALID_ARG, "NULL output");
    const int B = m->B, S = m->S, T = m->T;
    // block ranges: MM_RELAX_CTAS_PER_SM CTAs per SM over the scenario tiles,
    // at least one staged tile each
    const int zs = (S + kFwdSW - 1) / kFwdSW;
    const int nr = std::max(1, std::min((B + kFwdBT - 1) / kFwdBT, std::max(1, MM_RELAX_CTAS_PER_SM * m->num_sms / zs)));
    const size_t TS = (size_t)T * S;
    // scratch: range partials of O and V (FP32), then the terms in FP64
    st = relax_scratch(m, 2 * (size_t)nr * TS + 2 * TS);
    if (st != MM_OK) return st;
    float *part_o = m->relax_scratch, *part_v = part_o + (size_t)nr * TS;
    double *term = reinterpret_cast<double *>(part_v + (size_t)nr * TS);
    const RelaxEcon E = relax_econ(m, beta, m_ref);
    const RelaxRows Rw{m->val, m->R, m->ore_off};
    st = g_dev ? relax_fwd_launch<float>(x_dev, g_dev, Rw, m->mass, B, S, T, E, part_o, part_v, nr, m->stream)
               : relax_fwd_launch<double>(x_dev, m->grade, Rw, m->mass, B, S, T, E, part_o, part_v, nr, m->stream);
    if (st != MM_OK) return st;
    k_relax_finish<<<(unsigned)((TS + 31) / 32), 1024, 0, m->stream>>>(part_o, part_v, nr, S, T, m->disc, m->target, E,
                                                                       ore_t_dev, term, m->relax_tick, npv_dev, J_dev);
    return check_launch("k_relax_finish");
}

mm_status mm_relaxed_backward(mm_model *m, const float *x_dev, const float *g_dev, double beta, double m_ref,
                              const double *npv_dev, const double *ore_t_dev, const double *gJ_dev, float *gx_dev,
                              float *gg_dev) {
    mm_status st = relax_check(m, x_dev, beta, m_ref);
    if (st != MM_OK) return st;
    if (!npv_dev || !ore_t_dev || !gJ_dev || !gx_dev) return set_error(MM_ERR_INVALID_ARG, "NULL argument");
    const int B = m->B, S = m->S, T = m->T;
    const int Sp = S | 1;  // odd row stride of c
    st = relax_scratch(m, (size_t)S + (size_t)T * Sp);
    if (st != MM_OK) return st;
    float *w = m->relax_scratch, *c = w + S;
    const RelaxEcon E = relax_econ(m, beta, m_ref);
    // small CTAs: each forms the scenario mean and std itself, in FP64, so more
    // SMs share that work
    k_relax_coef<<<(unsigned)(((size_t)T * S + 63) / 64), 64, 0, m->stream>>>(npv_dev, ore_t_dev, m->target, gJ_dev, S,
                                                                               T, Sp, E, w, c);
    st = check_launch("k_relax_coef");
    if (st != MM_OK) return st;
    const RelaxRows Rw{m->val, m->R, m->ore_off};
    {
        // the tiled path, period tiles of up to kRelaxTile, when its shared memory fits
        const bool rows = g_dev == nullptr;
        size_t need = 0;
        for (int tb = 0; tb < T; tb += kRelaxTile) {
            const int tt = (std::min(kRelaxTile, T - tb) + 3) / 4 * 4;
            need = std::max(need, adj_layout(S, T, tt, rows).floats * sizeof(float));
        }
        if (need + 1024 <= (size_t)m->max_smem_optin) {
            const int tiles = (B + kAdjBT - 1) / kAdjBT;
            for (int tb = 0; tb < T; tb += kRelaxTile) {
                const int tt = (std::min(kRelaxTile, T - tb) + 3) / 4 * 4;
                const size_t sm = adj_layout(S, T, tt, rows).floats * sizeof(float);
                const void *fn = nullptr;
                switch (tt) {
#define MM_ADJ_CASE(V) case V: fn = rows ? (const void *)k_relax_adj_tiled<double, V> : (const void *)k_relax_adj_tiled<float, V>; break;
                    MM_ADJ_CASE(4) MM_ADJ_CASE(8) MM_ADJ_CASE(12) MM_ADJ_CASE(16) MM_ADJ_CASE(20) default: MM_ADJ_CASE(24)
#undef MM_ADJ_CASE
                }
                MM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm), "adjoint smem");
                int per_sm = 1;
                MM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * kAdjWarps, sm), "occupancy");
                const int grid = std::max(1, std::min(tiles, std::max(1, per_sm) * m->num_sms));
                void *args[] = {(void *)&x_dev, rows ? (void *)&m->grade : (void *)&g_dev, (void *)&Rw, (void *)&m->mass,
                                (void *)&w, (void *)&c, (void *)&m->disc, (void *)&B, (void *)&S, (void *)&T, (void *)&Sp,
                                (void *)&tb, (void *)&E, (void *)&gx_dev, (void *)&gg_dev};
                MM_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(32 * kAdjWarps), args, sm, m->stream), "adjoint launch");
            }
            return check_launch("k_relax_adj_tiled");
        }
    }
    const int W = (S + 31) / 32;
    const size_t smem = ((size_t)S + (size_t)T * Sp + 2 * (size_t)T) * sizeof(float) + (size_t)8 * W * sizeof(uint32_t);
    const void *fn = g_dev ? (const void *)k_relax_adjoint<float> : (const void *)k_relax_adjoint<double>;
    if (smem > 48 * 1024) {
        if (smem > (size_t)m->max_smem_optin) return set_error(MM_ERR_INVALID_ARG, "S x T too large for the adjoint");
        MM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "adjoint smem");
    }
    const int blocks = std::min((B + 7) / 8, m->num_sms * 8);
    if (g_dev)
        k_relax_adjoint<float><<<blocks, 256, smem, m->stream>>>(x_dev, g_dev, Rw, m->mass, w, c, m->disc, B, S, T, Sp,
                                                                 E, gx_dev, gg_dev);
    else
        k_relax_adjoint<double><<<blocks, 256, smem, m->stream>>>(x_dev, m->grade, Rw, m->mass, w, c, m->disc, B, S, T,
                                                                  Sp, E, gx_dev, gg_dev);
    return check_launch("k_relax_adjoint");
}

}  // extern "C"
