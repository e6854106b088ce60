// Relaxed objective: forward and hand-written adjoint.
//
// The extraction decision x[b][t] of Eq. 14 relaxed to [0, 1], the mill
// penalty smoothed by a softplus of width m_ref / beta, and the risk term
// J = mean_s NPV_s - lambda std_s NPV_s:
//   O[t][s] = sum_b x[b][t] m_b ore[b][s],   V[t][s] = sum_b x[b][t] v[b][s],
//   NPV_s   = sum_t d_t (V[t][s] - P_t(O[t][s])),
//   P_t(O)  = a m_ref sp((Q_t - O) / m_ref) + e m_ref sp((O - Q_t) / m_ref),
//   sp(z)   = log(1 + exp(beta z)) / beta.
// ore and v come from the grades g exactly as in the discrete model (the ore
// decision in FP64 on the given grade values; v in FP32); ore is a step in g
// and carries no gradient.
//
// Forward: the two skinny contractions over blocks run on CUDA cores -- each
// CTA takes a chunk of blocks and a tile of periods, one thread per scenario,
// FP32 products summed over the chunk -- and the chunk partials are added in
// FP64 in chunk order (deterministic).  O[t][s] is kept as the checkpoint the
// adjoint reads, so the backward pass never redoes the contraction.
// Adjoint: with w_s = dJ/dNPV_s and c[t][s] = w_s P_t'(O[t][s]),
//   dJ/dx[b][t] = d_t (sum_s w_s v[b][s] - m_b sum_s c[t][s] ore[b][s]),
//   dJ/dg[b][s] = w_s ore[b][s] m_b price recovery sum_t d_t x[b][t],
// one warp per block.
#include <algorithm>
#include <cmath>

#include "mm_internal.cuh"

namespace mm {

constexpr int kRelaxChunk = 128;  // blocks per forward CTA
constexpr int kRelaxTile = 16;    // periods per forward CTA

struct RelaxEcon {
    double p, r, pc;   // price, recovery, processing cost (FP64 ore decision)
    float pf, rf, pcf, mcf;
    double a, e, lambda, beta, m_ref;
};

template <typename G>
__device__ __forceinline__ bool relax_ore(G g, const RelaxEcon &E) {
    return ((double)g * E.p) * E.r > E.pc;
}

// v in FP32: m ((g price) recovery - pc) - m mc for ore, -m mc for waste.
template <typename G>
__device__ __forceinline__ float relax_value(G g, bool ore, float m, const RelaxEcon &E) {
    const float mc = m * E.mcf;
    return ore ? m * (((float)g * E.pf) * E.rf - E.pcf) - mc : -mc;
}

// Partial sums of O and V over one chunk of blocks for one tile of periods.
template <typename G>
__global__ void __launch_bounds__(1024) k_relax_partial(const float *__restrict__ x, const G *__restrict__ g,
                                                        const uint32_t *__restrict__ mass, int32_t B, int32_t S,
                                                        int32_t T, RelaxEcon E, float *__restrict__ part_o,
                                                        float *__restrict__ part_v) {
    __shared__ float s_x[kRelaxChunk][kRelaxTile];
    __shared__ float s_m[kRelaxChunk];
    const int chunk = blockIdx.x, t0 = blockIdx.y * kRelaxTile;
    const int b0 = chunk * kRelaxChunk;
    const int nb = min(kRelaxChunk, B - b0), nt = min(kRelaxTile, T - t0);
    for (int i = threadIdx.x; i < kRelaxChunk * kRelaxTile; i += blockDim.x) {
        const int bb = i / kRelaxTile, j = i % kRelaxTile;
        s_x[bb][j] = (bb < nb && j < nt) ? x[(size_t)(b0 + bb) * T + t0 + j] : 0.0f;
    }
    for (int i = threadIdx.x; i < kRelaxChunk; i += blockDim.x) s_m[i] = i < nb ? (float)mass[b0 + i] : 0.0f;
    __syncthreads();
    const int s = threadIdx.x;
    if (s >= S) return;
    float o[kRelaxTile], v[kRelaxTile];
#pragma unroll
    for (int j = 0; j < kRelaxTile; j++) o[j] = v[j] = 0.0f;
    for (int bb = 0; bb < nb; bb++) {
        const G gv = g[(size_t)(b0 + bb) * S + s];
        const bool ore = relax_ore(gv, E);
        const float m = s_m[bb];
        const float val = relax_value(gv, ore, m, E);
        const float mo = ore ? m : 0.0f;
#pragma unroll
        for (int j = 0; j < kRelaxTile; j++) {
            const float xv = s_x[bb][j];
            o[j] = fmaf(xv, mo, o[j]);
            v[j] = fmaf(xv, val, v[j]);
        }
    }
    for (int j = 0; j < nt; j++) {
        const size_t i = ((size_t)chunk * T + t0 + j) * S + s;
        part_o[i] = o[j];
        part_v[i] = v[j];
    }
}

// O and V from the chunk partials, added in FP64 in chunk order.
__global__ void k_relax_reduce(const float *__restrict__ part_o, const float *__restrict__ part_v, int32_t nchunks,
                               int32_t TS, double *__restrict__ o_out, double *__restrict__ v_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TS) return;
    double so = 0.0, sv = 0.0;
    for (int c = 0; c < nchunks; c++) {
        so += (double)part_o[(size_t)c * TS + i];
        sv += (double)part_v[(size_t)c * TS + i];
    }
    o_out[i] = so;
    v_out[i] = sv;
}

__device__ __forceinline__ double relax_softplus(double z, double beta) {
    const double bz = beta * z;
    return (fmax(bz, 0.0) + log1p(exp(-fabs(bz)))) / beta;
}
__device__ __forceinline__ double relax_sigmoid(double z, double beta) { return 1.0 / (1.0 + exp(-beta * z)); }

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

// NPV_s and J (one CTA, one thread per scenario).
__global__ void __launch_bounds__(1024) k_relax_npv(const double *__restrict__ o, const double *__restrict__ v,
                                                    const double *__restrict__ disc, const uint64_t *__restrict__ target,
                                                    int32_t S, int32_t T, RelaxEcon E, double *__restrict__ npv,
                                                    double *__restrict__ J) {
    __shared__ double red[33];
    const int s = threadIdx.x;
    double acc = 0.0;
    if (s < S) {
        for (int t = 0; t < T; t++) {
            const double O = o[(size_t)t * S + s], Q = (double)target[t];
            const double pen = E.a * E.m_ref * relax_softplus((Q - O) / E.m_ref, E.beta) +
                               E.e * E.m_ref * relax_softplus((O - Q) / E.m_ref, E.beta);
            acc += disc[t] * (v[(size_t)t * S + s] - pen);
        }
        npv[s] = acc;
    }
    const double mean = relax_block_sum(s < S ? acc : 0.0, red) / S;
    const double dv = s < S ? acc - mean : 0.0;
    const double var = relax_block_sum(dv * dv, red) / S;
    if (s == 0) J[0] = mean - E.lambda * sqrt(var);
}

// Adjoint coefficients: w_s = gJ (1/S - lambda (NPV_s - mean) / (S std))
// (the std term dropped where std = 0) and c[t][s] = w_s P_t'(O[t][s]).
__global__ void __launch_bounds__(1024) k_relax_coef(const double *__restrict__ npv, const double *__restrict__ o,
                                                     const uint64_t *__restrict__ target, const double *__restrict__ gJ,
                                                     int32_t S, int32_t T, int32_t Sp, RelaxEcon E,
                                                     float *__restrict__ w_out, float *__restrict__ c_out) {
    __shared__ double red[33];
    const int s = threadIdx.x;
    const double x = s < S ? npv[s] : 0.0;
    const double mean = relax_block_sum(x, red) / S;
    const double dv = s < S ? x - mean : 0.0;
    const double sd = sqrt(relax_block_sum(dv * dv, red) / S);
    if (s >= S) return;
    const double g = gJ[0];
    double w = g / S;
    if (sd > 0.0) w -= g * E.lambda * dv / (S * sd);
    w_out[s] = (float)w;
    for (int t = 0; t < T; t++) {
        const double O = o[(size_t)t * S + s], Q = (double)target[t];
        const double dp = -E.a * relax_sigmoid((Q - O) / E.m_ref, E.beta) + E.e * relax_sigmoid((O - Q) / E.m_ref, E.beta);
        c_out[(size_t)t * Sp + s] = (float)(w * dp);
    }
}

// dJ/dx and dJ/dg, one warp per block.  Shared memory: w[S], c[T][Sp] (Sp odd:
// lane t reads row t without bank conflicts), d[T], the warp's ore bits.
template <typename G>
__global__ void __launch_bounds__(256) k_relax_adjoint(const float *__restrict__ x, const G *__restrict__ g,
                                                       const uint32_t *__restrict__ mass, const float *__restrict__ w,
                                                       const float *__restrict__ c, const double *__restrict__ disc,
                                                       int32_t B, int32_t S, int32_t T, int32_t Sp, RelaxEcon E,
                                                       float *__restrict__ gx, float *__restrict__ gg) {
    extern __shared__ __align__(16) float s_relax[];
    const int W = (S + 31) / 32;
    float *s_w = s_relax;                              // [S]
    float *s_c = s_w + S;                              // [T][Sp]
    float *s_d = s_c + (size_t)T * Sp;                 // [T]
    uint32_t *s_ore = reinterpret_cast<uint32_t *>(s_d + T);  // [warps][W]
    for (int i = threadIdx.x; i < S; i += blockDim.x) s_w[i] = w[i];
    for (int i = threadIdx.x; i < T * Sp; i += blockDim.x) s_c[i] = c[i];
    for (int i = threadIdx.x; i < T; i += blockDim.x) s_d[i] = (float)disc[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *ore_w = s_ore + (size_t)warp * W;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const float prf = E.pf * E.rf;
    for (int b = blockIdx.x * (blockDim.x >> 5) + warp; b < B; b += nwarps) {
        const float m = (float)mass[b];
        // u = sum_s w_s v[b][s]; ore bits of the block
        float u = 0.0f;
        for (int s0 = 0; s0 < S; s0 += 32) {
            const int s = s0 + lane;
            bool ore = false;
            if (s < S) {
                const G gv = g[(size_t)b * S + s];
                ore = relax_ore(gv, E);
                u = fmaf(s_w[s], relax_value(gv, ore, m, E), u);
            }
            const uint32_t bits = __ballot_sync(0xffffffffu, ore);
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
        // dJ/dx: lane t sums c[t][s] over the ore scenarios
        for (int t = lane; t < T; t += 32) {
            const float *crow = s_c + (size_t)t * Sp;
            float acc = 0.0f;
            for (int k = 0; k < W; k++) {
                uint32_t bits = ore_w[k];
                while (bits) {
                    const int j = __ffs(bits) - 1;
                    bits &= bits - 1;
                    acc += crow[k * 32 + j];
                }
            }
            gx[(size_t)b * T + t] = s_d[t] * (u - m * acc);
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

static RelaxEcon relax_econ(const mm_model *m, double beta, double m_ref) {
    RelaxEcon E;
    E.p = m->price; E.r = m->recovery; E.pc = m->proc_cost;
    E.pf = (float)m->price; E.rf = (float)m->recovery; E.pcf = (float)m->proc_cost; E.mcf = (float)m->mining_cost;
    E.a = m->shortfall_pen; E.e = m->excess_pen; E.lambda = m->lambda; E.beta = beta; E.m_ref = m_ref;
    return E;
}

static mm_status relax_check(mm_model *m, const float *x, double beta, double m_ref) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
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
    // scratch: chunk partials of O and V (FP32), then V in FP64
    st = relax_scratch(m, 2 * (size_t)nchunks * TS + 2 * TS);
    if (st != MM_OK) return st;
    float *part_o = m->relax_scratch, *part_v = part_o + (size_t)nchunks * TS;
    double *v_sum = reinterpret_cast<double *>(part_v + (size_t)nchunks * TS);
    const RelaxEcon E = relax_econ(m, beta, m_ref);
    const dim3 grid(nchunks, (T + kRelaxTile - 1) / kRelaxTile);
    const int threads = ((S + 31) / 32) * 32;
    if (g_dev)
        k_relax_partial<float><<<grid, threads, 0, m->stream>>>(x_dev, g_dev, m->mass, B, S, T, E, part_o, part_v);
    else
        k_relax_partial<double><<<grid, threads, 0, m->stream>>>(x_dev, m->grade, m->mass, B, S, T, E, part_o, part_v);
    st = check_launch("k_relax_partial");
    if (st != MM_OK) return st;
    k_relax_reduce<<<(unsigned)((TS + 255) / 256), 256, 0, m->stream>>>(part_o, part_v, nchunks, (int)TS, ore_t_dev,
                                                                       v_sum);
    st = check_launch("k_relax_reduce");
    if (st != MM_OK) return st;
    k_relax_npv<<<1, threads, 0, m->stream>>>(ore_t_dev, v_sum, m->disc, m->target, S, T, E, npv_dev, J_dev);
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
    const int threads = ((S + 31) / 32) * 32;
    k_relax_coef<<<1, threads, 0, m->stream>>>(npv_dev, ore_t_dev, m->target, gJ_dev, S, T, Sp, E, w, c);
    st = check_launch("k_relax_coef");
    if (st != MM_OK) return st;
    const int W = (S + 31) / 32;
    const size_t smem = ((size_t)S + (size_t)T * Sp + T) * sizeof(float) + (size_t)8 * W * sizeof(uint32_t);
    const void *fn = g_dev ? (const void *)k_relax_adjoint<float> : (const void *)k_relax_adjoint<double>;
    if (smem > 48 * 1024) {
        if (smem > (size_t)m->max_smem_optin) return set_error(MM_ERR_INVALID_ARG, "S x T too large for the adjoint");
        MM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "adjoint smem");
    }
    const int blocks = std::min((B + 7) / 8, m->num_sms * 8);
    if (g_dev)
        k_relax_adjoint<float><<<blocks, 256, smem, m->stream>>>(x_dev, g_dev, m->mass, w, c, m->disc, B, S, T, Sp, E,
                                                                 gx_dev, gg_dev);
    else
        k_relax_adjoint<double><<<blocks, 256, smem, m->stream>>>(x_dev, m->grade, m->mass, w, c, m->disc, B, S, T, Sp,
                                                                  E, gx_dev, gg_dev);
    return check_launch("k_relax_adjoint");
}

}  // extern "C"
