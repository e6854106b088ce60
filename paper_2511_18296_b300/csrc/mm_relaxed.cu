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

constexpr int kRelaxChunk = 128;  // blocks per forward CTA
constexpr int kRelaxTile = 24;    // periods per forward CTA (at most; wider tiles spill)

struct RelaxEcon {
    double p, r, pc;   // price, recovery, processing cost (FP64 ore decision)
    float pf, rf, pcf, mcf;
    double a, e, lambda, beta, m_ref;
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

// Raw inputs of (b, s) for relax_eval: the grade (caller grades) or the value
// and ore word from the model's rows (model grades); fetched ahead of use.
struct RelaxRaw {
    float a;
    uint32_t w;
};
template <typename G>
__device__ __forceinline__ RelaxRaw relax_fetch(const G *g, const RelaxRows &Rw, int32_t b, int32_t S, int s);
template <>
__device__ __forceinline__ RelaxRaw relax_fetch<float>(const float *g, const RelaxRows &, int32_t b, int32_t S, int s) {
    return RelaxRaw{__ldg(g + (size_t)b * S + s), 0u};
}
template <>
__device__ __forceinline__ RelaxRaw relax_fetch<double>(const double *, const RelaxRows &Rw, int32_t b, int32_t,
                                                        int s) {
    const float *row = Rw.val + (size_t)b * Rw.R;
    return RelaxRaw{__ldg(row + s), __ldg(reinterpret_cast<const uint32_t *>(row + Rw.ore_off) + (s >> 5))};
}
template <typename G>
__device__ __forceinline__ void relax_eval(RelaxRaw r, int s, float m, const RelaxEcon &E, bool &ore, float &val);
template <>
__device__ __forceinline__ void relax_eval<float>(RelaxRaw r, int, float m, const RelaxEcon &E, bool &ore, float &val) {
    ore = relax_ore(r.a, E);
    const float mc = m * E.mcf;
    val = ore ? m * ((r.a * E.pf) * E.rf - E.pcf) - mc : -mc;
}
template <>
__device__ __forceinline__ void relax_eval<double>(RelaxRaw r, int s, float, const RelaxEcon &, bool &ore, float &val) {
    val = r.a;
    ore = (r.w >> (s & 31)) & 1u;
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

// Partial sums of O and V over one chunk of blocks for one tile of TT periods
// starting at t_base (TT a multiple of 4: the staged x rows are read four
// periods at a time).  Thread (s, k): scenario blockIdx.z * SW + s,
// blocks k, k + KS, ... of the chunk; the KS partial sums of a scenario are
// then added in k order through shared memory (deterministic), so KS times
// more warps keep loads in flight than one thread per scenario would.
constexpr int kRelaxSplit = 4;
template <typename G, int TT>
__global__ void __launch_bounds__(512) k_relax_partial(const float *__restrict__ x, const G *__restrict__ g,
                                                        RelaxRows Rw, const uint32_t *__restrict__ mass, int32_t B,
                                                        int32_t S, int32_t T, int32_t t_base, RelaxEcon E,
                                                        float *__restrict__ part_o, float *__restrict__ part_v) {
    constexpr int KS = kRelaxSplit;
    __shared__ __align__(16) float s_x[kRelaxChunk][TT];
    __shared__ float s_m[kRelaxChunk];
    extern __shared__ float s_red[];  // [KS - 1][TT][SW]
    const int SW = blockDim.x / KS;   // scenarios per CTA
    const int chunk = blockIdx.x, t0 = t_base;
    const int b0 = chunk * kRelaxChunk;
    const int nb = min(kRelaxChunk, B - b0), nt = min(TT, T - t0);
    for (int i = threadIdx.x; i < kRelaxChunk * TT; i += blockDim.x) {
        const int bb = i / TT, j = i % TT;
        s_x[bb][j] = (bb < nb && j < nt) ? x[(size_t)(b0 + bb) * T + t0 + j] : 0.0f;
    }
    for (int i = threadIdx.x; i < kRelaxChunk; i += blockDim.x) s_m[i] = i < nb ? (float)mass[b0 + i] : 0.0f;
    __syncthreads();
    const int sl = threadIdx.x % SW, k = threadIdx.x / SW;
    const int s = blockIdx.z * SW + sl;
    const bool live = s < S;
    float o[TT], v[TT];
#pragma unroll
    for (int j = 0; j < TT; j++) o[j] = v[j] = 0.0f;
    if (live) {
        // two blocks' inputs in flight ahead of use
        RelaxRaw r0 = k < nb ? relax_fetch<G>(g, Rw, b0 + k, S, s) : RelaxRaw{0.0f, 0u};
        RelaxRaw r1 = k + KS < nb ? relax_fetch<G>(g, Rw, b0 + k + KS, S, s) : RelaxRaw{0.0f, 0u};
        for (int bb = k; bb < nb; bb += KS) {
            const RelaxRaw rc = r0;
            r0 = r1;
            if (bb + 2 * KS < nb) r1 = relax_fetch<G>(g, Rw, b0 + bb + 2 * KS, S, s);
            bool ore;
            float val;
            relax_eval<G>(rc, s, s_m[bb], E, ore, val);
            const float mo = ore ? s_m[bb] : 0.0f;
            const float4 *xr = reinterpret_cast<const float4 *>(s_x[bb]);
#pragma unroll
            for (int q = 0; q < TT / 4; q++) {
                const float4 x4 = xr[q];
                o[4 * q] = fmaf(x4.x, mo, o[4 * q]);
                o[4 * q + 1] = fmaf(x4.y, mo, o[4 * q + 1]);
                o[4 * q + 2] = fmaf(x4.z, mo, o[4 * q + 2]);
                o[4 * q + 3] = fmaf(x4.w, mo, o[4 * q + 3]);
                v[4 * q] = fmaf(x4.x, val, v[4 * q]);
                v[4 * q + 1] = fmaf(x4.y, val, v[4 * q + 1]);
                v[4 * q + 2] = fmaf(x4.z, val, v[4 * q + 2]);
                v[4 * q + 3] = fmaf(x4.w, val, v[4 * q + 3]);
            }
        }
    }
    // o: partials of k >= 1 to shared memory, k = 0 adds them in k order; then
    // v.  Written out twice with static indices so o and v stay in registers.
    if (k > 0) {
#pragma unroll
        for (int j = 0; j < TT; j++) s_red[((size_t)(k - 1) * TT + j) * SW + sl] = o[j];
    }
    __syncthreads();
    if (k == 0 && live) {
#pragma unroll
        for (int j = 0; j < TT; j++) {
            float a = o[j];
#pragma unroll
            for (int kk = 1; kk < KS; kk++) a += s_red[((size_t)(kk - 1) * TT + j) * SW + sl];
            if (j < nt) part_o[((size_t)chunk * T + t0 + j) * S + s] = a;
        }
    }
    __syncthreads();
    if (k > 0) {
#pragma unroll
        for (int j = 0; j < TT; j++) s_red[((size_t)(k - 1) * TT + j) * SW + sl] = v[j];
    }
    __syncthreads();
    if (k == 0 && live) {
#pragma unroll
        for (int j = 0; j < TT; j++) {
            float a = v[j];
#pragma unroll
            for (int kk = 1; kk < KS; kk++) a += s_red[((size_t)(kk - 1) * TT + j) * SW + sl];
            if (j < nt) part_v[((size_t)chunk * T + t0 + j) * S + s] = a;
        }
    }
}

template <typename G, int TT>
static void relax_partial_tile(dim3 grid, int threads, size_t smem, cudaStream_t st, const float *x, const G *g,
                               RelaxRows Rw, const uint32_t *mass, int32_t B, int32_t S, int32_t T, int32_t tb,
                               RelaxEcon E, float *part_o, float *part_v) {
    // static + dynamic shared memory passes 48 KB for the wide tiles
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_relax_partial<G, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)((kRelaxSplit - 1) * TT * (512 / kRelaxSplit) * sizeof(float)));
    (void)attr;
    k_relax_partial<G, TT><<<grid, threads, smem, st>>>(x, g, Rw, mass, B, S, T, tb, E, part_o, part_v);
}

template <typename G>
static mm_status relax_partial_launch(const float *x, const G *g, RelaxRows Rw, const uint32_t *mass, int32_t B,
                                      int32_t S, int32_t T, RelaxEcon E, float *part_o, float *part_v, int nchunks,
                                      int threads, cudaStream_t st) {
    // tiles of up to kRelaxTile periods, each as wide as needed rounded up to 4,
    // so a batch with T <= kRelaxTile reads the grades once
    const int sw = threads / kRelaxSplit;
    const int zs = (S + sw - 1) / sw;
    for (int tb = 0; tb < T; tb += kRelaxTile) {
        const int w = std::min(kRelaxTile, T - tb), tt = (w + 3) / 4 * 4;
        const dim3 grid(nchunks, 1, zs);
        const size_t smem = (size_t)(kRelaxSplit - 1) * tt * sw * sizeof(float);
        switch (tt) {
            case 4: relax_partial_tile<G, 4>(grid, threads, smem, st, x, g, Rw, mass, B, S, T, tb, E, part_o, part_v); break;
            case 8: relax_partial_tile<G, 8>(grid, threads, smem, st, x, g, Rw, mass, B, S, T, tb, E, part_o, part_v); break;
            case 12: relax_partial_tile<G, 12>(grid, threads, smem, st, x, g, Rw, mass, B, S, T, tb, E, part_o, part_v); break;
            case 16: relax_partial_tile<G, 16>(grid, threads, smem, st, x, g, Rw, mass, B, S, T, tb, E, part_o, part_v); break;
            case 20: relax_partial_tile<G, 20>(grid, threads, smem, st, x, g, Rw, mass, B, S, T, tb, E, part_o, part_v); break;
            default: relax_partial_tile<G, 24>(grid, threads, smem, st, x, g, Rw, mass, B, S, T, tb, E, part_o, part_v); break;
        }
        mm_status r = check_launch("k_relax_partial");
        if (r != MM_OK) return r;
    }
    return MM_OK;
}

// O and V from the chunk partials in FP64, one warp per (t, s): lane l adds
// chunks l, l + 32, ... in order, then a fixed xor tree (deterministic).
__global__ void __launch_bounds__(256) k_relax_reduce(const float *__restrict__ part_o,
                                                      const float *__restrict__ part_v, int32_t nchunks, int32_t TS,
                                                      double *__restrict__ o_out, double *__restrict__ v_out) {
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= TS) return;
    double so = 0.0, sv = 0.0;
    for (int c = lane; c < nchunks; c += 32) {
        so += (double)__ldg(part_o + (size_t)c * TS + i);
        sv += (double)__ldg(part_v + (size_t)c * TS + i);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        so += __shfl_xor_sync(0xffffffffu, so, off);
        sv += __shfl_xor_sync(0xffffffffu, sv, off);
    }
    if (lane == 0) {
        o_out[i] = so;
        v_out[i] = sv;
    }
}

// softplus and its derivative of beta z, the argument formed in FP64 and the
// transcendental part in FP32 (relative error ~1e-7 of a term far below the
// NPV and gradient tolerances).
__device__ __forceinline__ double relax_softplus(double z, double beta) {
    const double bz = beta * z;
    const float abz = (float)fabs(bz);
    return (fmax(bz, 0.0) + (double)log1pf(expf(-abz))) / beta;
}
__device__ __forceinline__ double relax_sigmoid(double z, double beta) {
    return (double)(1.0f / (1.0f + expf((float)(-beta * z))));
}

// FP64 sum over the threads of one CTA (valid in every thread).
__device__ double relax_block_sum(double x, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; w++) t += red[w];
        red[32] = t;
    }
    __syncthreads();
    const double r = red[32];
    __syncthreads();
    return r;
}

// Discounted net value of every (t, s): d_t (V[t][s] - P_t(O[t][s])), one
// thread each over many CTAs (FP64 is scarce per SM on this part).
__global__ void __launch_bounds__(256) k_relax_terms(const double *__restrict__ o, const double *__restrict__ v,
                                                     const double *__restrict__ disc,
                                                     const uint64_t *__restrict__ target, int32_t S, int32_t TS,
                                                     RelaxEcon E, double *__restrict__ term) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TS) return;
    const int t = i / S;
    const double O = o[i], Q = (double)target[t], inv = 1.0 / E.m_ref;
    const double pen = E.a * E.m_ref * relax_softplus((Q - O) * inv, E.beta) +
                       E.e * E.m_ref * relax_softplus((O - Q) * inv, E.beta);
    term[i] = disc[t] * (v[i] - pen);
}

// NPV_s = sum_t term[t][s] (period order) and J (one CTA, one thread per scenario).
__global__ void __launch_bounds__(1024) k_relax_npv(const double *__restrict__ term, int32_t S, int32_t T,
                                                    RelaxEcon E, double *__restrict__ npv, double *__restrict__ J) {
    __shared__ double red[33];
    const int s = threadIdx.x;
    double acc = 0.0;
    if (s < S) {
        for (int t = 0; t < T; t++) acc += term[(size_t)t * S + s];
        npv[s] = acc;
    }
    const double mean = relax_block_sum(s < S ? acc : 0.0, red) / S;
    const double dv = s < S ? acc - mean : 0.0;
    const double var = relax_block_sum(dv * dv, red) / S;
    if (s == 0) J[0] = mean - E.lambda * sqrt(var);
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
    const double mean = relax_block_sum(part, red) / S;
    double pv = 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double d = npv[s] - mean;
        pv += d * d;
    }
    const double sd = sqrt(relax_block_sum(pv, red) / S);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= T * S) return;
    const int t = i / S, s = i - t * S;
    const double g = gJ[0];
    double w = g / S;
    if (sd > 0.0) w -= g * E.lambda * (npv[s] - mean) / (S * sd);
    if (t == 0) w_out[s] = (float)w;
    const double O = o[i], Q = (double)target[t], inv = 1.0 / E.m_ref;
    const double dp = -E.a * relax_sigmoid((Q - O) * inv, E.beta) + E.e * relax_sigmoid((O - Q) * inv, E.beta);
    c_out[(size_t)t * Sp + s] = (float)(w * dp);
}

// dJ/dx and dJ/dg, one warp per block.  Shared memory: w[S], c[T][Sp] (Sp odd:
// lane t reads row t without bank conflicts), d[T], the warp's ore bits.
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

}  // namespace mm

using namespace mm;

extern "C" {

mm_status mm_relaxed_forward(mm_model *m, const float *x_dev, const float *g_dev, double beta, double m_ref,
                             double *J_dev, double *npv_dev, double *ore_t_dev) {
    mm_status st = relax_check(m, x_dev, beta, m_ref);
    if (st != MM_OK) return st;
    if (!J_dev || !npv_dev || !ore_t_dev) return set_error(MM_ERR_INVALID_ARG, "NULL output");
    const int B = m->B, S = m->S, T = m->T;
    const int nchunks = (B + kRelaxChunk - 1) / kRelaxChunk;
    const size_t TS = (size_t)T * S;
    // scratch: chunk partials of O and V (FP32), then V and the terms in FP64
    st = relax_scratch(m, 2 * (size_t)nchunks * TS + 4 * TS);
    if (st != MM_OK) return st;
    float *part_o = m->relax_scratch, *part_v = part_o + (size_t)nchunks * TS;
    double *v_sum = reinterpret_cast<double *>(part_v + (size_t)nchunks * TS);
    const RelaxEcon E = relax_econ(m, beta, m_ref);
    const int threads = kRelaxSplit * std::min(((S + 31) / 32) * 32, 128);  // scenarios per CTA x split
    const RelaxRows Rw{m->val, m->R, m->ore_off};
    st = g_dev ? relax_partial_launch<float>(x_dev, g_dev, Rw, m->mass, B, S, T, E, part_o, part_v, nchunks, threads,
                                             m->stream)
               : relax_partial_launch<double>(x_dev, m->grade, Rw, m->mass, B, S, T, E, part_o, part_v, nchunks,
                                              threads, m->stream);
    if (st != MM_OK) return st;
    k_relax_reduce<<<(unsigned)((TS * 32 + 255) / 256), 256, 0, m->stream>>>(part_o, part_v, nchunks, (int)TS,
                                                                            ore_t_dev, v_sum);
    st = check_launch("k_relax_reduce");
    if (st != MM_OK) return st;
    double *term = v_sum + TS;
    k_relax_terms<<<(unsigned)((TS + 255) / 256), 256, 0, m->stream>>>(ore_t_dev, v_sum, m->disc, m->target, S, (int)TS,
                                                                      E, term);
    st = check_launch("k_relax_terms");
    if (st != MM_OK) return st;
    k_relax_npv<<<1, ((S + 31) / 32) * 32, 0, m->stream>>>(term, S, T, E, npv_dev, J_dev);  // a thread per scenario
    return check_launch("k_relax_npv");
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
    k_relax_coef<<<(unsigned)(((size_t)T * S + 255) / 256), 256, 0, m->stream>>>(npv_dev, ore_t_dev, m->target,
                                                                                  gJ_dev, S, T, Sp, E, w, c);
    st = check_launch("k_relax_coef");
    if (st != MM_OK) return st;
    const int W = (S + 31) / 32;
    const size_t smem = ((size_t)S + (size_t)T * Sp + 2 * (size_t)T) * sizeof(float) + (size_t)8 * W * sizeof(uint32_t);
    const void *fn = g_dev ? (const void *)k_relax_adjoint<float> : (const void *)k_relax_adjoint<double>;
    if (smem > 48 * 1024) {
        if (smem > (size_t)m->max_smem_optin) return set_error(MM_ERR_INVALID_ARG, "S x T too large for the adjoint");
        MM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "adjoint smem");
    }
    const int blocks = std::min((B + 7) / 8, m->num_sms * 8);
    const RelaxRows Rw{m->val, m->R, m->ore_off};
    if (g_dev)
        k_relax_adjoint<float><<<blocks, 256, smem, m->stream>>>(x_dev, g_dev, Rw, m->mass, w, c, m->disc, B, S, T, Sp,
                                                                 E, gx_dev, gg_dev);
    else
        k_relax_adjoint<double><<<blocks, 256, smem, m->stream>>>(x_dev, m->grade, Rw, m->mass, w, c, m->disc, B, S, T,
                                                                  Sp, E, gx_dev, gg_dev);
    return check_launch("k_relax_adjoint");
}

}  // extern "C"
