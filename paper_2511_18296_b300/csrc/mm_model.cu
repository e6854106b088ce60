// Model store, schedule state and the apply-move kernel.
//
// Device layout (per model):
//   val   [B+1][R]          one combined row per block, R = roundup(4*ceil(S/4) + W, 8)
//                           floats (32-byte multiple): S FP32 values (scenario
//                           fastest), zeros up to ore_off = 4*ceil(S/4), then
//                           W = ceil(S/32) ore words (bit s%32 of word s/32), zeros;
//                           a moved block is one contiguous gather (one bulk copy);
//                           row B is all zeros (the stand-in partner of a shift)
//   blk   u32  [B]          packed period | lo << 8 | hi << 16
//   grade FP64 [B][S]       kept for the FP64 metal accumulators
//   minedT i64 [T+1], oreT i64 [T+1][S], metal FP64 [T][S], npv FP64 [S]
//   contrib FP64 [T][S]     d_t (cash_t,s - pen_t,s): NPV_s = sum_t contrib[t][s]
//   tab   FP32 [2][T+1][S_pad]  NPV change of removing / adding one block of ore
//   ctab  FP32 [T+1][T+1][S_pad] Pout[a] + Pin[b]: the penalty change of moving one
//         block of ore from period a to period b (kept while T <= kCtabMaxT)
//                               in period t, scenario s (uniform block mass)
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <numeric>

#include "mm_apply.cuh"

namespace mm {

static thread_local char g_err[512] = "";

mm_status set_error(mm_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

mm_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(MM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(MM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

mm_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, what);
    return MM_OK;
}

mm_status read_sticky(mm_model *m) {
    MM_CUDA_TRY(cudaMemcpyAsync(m->status_host, m->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, m->stream),
                "read status");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    return sticky_status(m, *m->status_host);
}

// Map the sticky bits st (already read back) to a status and clear them.
mm_status sticky_status(mm_model *m, uint32_t st) {
    if (st) {
        MM_CUDA_TRY(cudaMemsetAsync(m->status, 0, sizeof(uint32_t), m->stream), "clear status");
        if (st & kStTimeout) return set_error(MM_ERR_TIMEOUT, "a bounded device wait ran out");
        if (st & kStBadMove) return set_error(MM_ERR_BAD_MOVE, "a batch contained a move with a block or period out of range");
    }
    return MM_OK;
}

static Topo topo_of(const mm_model *m) {
    Topo tp;
    tp.B = m->B; tp.T = m->T; tp.nx = m->nx; tp.ny = m->ny; tp.nz = m->nz;
    tp.pred_ptr = m->pred_ptr; tp.pred_idx = m->pred_idx; tp.succ_ptr = m->succ_ptr; tp.succ_idx = m->succ_idx;
    return tp;
}

Topo topo_of_model(const mm_model *m) { return topo_of(m); }

// ---------------------------------------------------------------- kernels

// Ore/waste and FP32 value rows.  One thread per (block, ore word): 32
// scenarios.  FP64 with explicit round-to-nearest operations in the order
// ((g*price)*recovery) > proc_cost; value = m*(rev - pc) - m*mc or -(m*mc).
// margin_only (uncertainty weights present): the row holds the processing
// margin m*(rev - pc) of an ore scenario and 0 for waste, the part that
// sigma(s,t) scales (Eq. 12); the mining cost is added per move.
__global__ void k_classify(const double *__restrict__ grade, const uint32_t *__restrict__ mass, int32_t B, int32_t S,
                           int32_t R, int32_t ore_off, int32_t W, double price, double recovery, double pc,
                           double mc, int margin_only, float *__restrict__ val) {
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)B * W) return;
    int32_t b = (int32_t)(gid / W), w = (int32_t)(gid % W);
    double m = (double)mass[b];
    float *row = val + (int64_t)b * R;
    uint32_t bits = 0;
    for (int j = 0; j < 32; j++) {
        int s = w * 32 + j;
        if (s >= S) break;
        double g = grade[(int64_t)b * S + s];
        double rev = __dmul_rn(__dmul_rn(g, price), recovery);
        bool o = rev > pc;
        double vv;
        if (margin_only) vv = o ? __dmul_rn(m, __dsub_rn(rev, pc)) : 0.0;
        else vv = o ? __dsub_rn(__dmul_rn(m, __dsub_rn(rev, pc)), __dmul_rn(m, mc)) : -__dmul_rn(m, mc);
        row[s] = __double2float_rn(vv);
        bits |= (o ? 1u : 0u) << j;
    }
    reinterpret_cast<uint32_t *>(row + ore_off)[w] = bits;
}

// Packed period/lo/hi word of every block.
__global__ void k_blk_build(Topo tp, const uint8_t *__restrict__ period, uint32_t *__restrict__ blk) {
    int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= tp.B) return;
    blk[b] = block_bounds(tp, b, [&](int32_t j) { return (uint32_t)period[j]; });
}

// Base feasibility: every arc p -> b with x_p <= x_b (checked from lo_b).
__global__ void k_base_arcs(int32_t B, const uint32_t *__restrict__ blk, uint32_t *__restrict__ bad) {
    int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    uint32_t w = blk[b];
    if (blk_lo(w) > blk_period(w)) atomicOr(bad, 1u);
}

// Per-period sums in a fixed order (blocks of period t sorted by id), in two
// levels.  k_accum_part: one CTA per chunk of up to accum_chunk_len
// consecutive blocks of one period (chunk table built on the host); thread s
// sums scenario s over the chunk's blocks, eight blocks' loads in flight at a
// time: ore tonnage (integer), metal m_b * g[b][s] of ore blocks (FP64, block
// order) and, in thread 0, the mined tonnage.  k_accum_reduce: for period t
// and 32 scenarios, warp u adds every eighth chunk partial from chunk u on, in
// chunk order, and the eight warps' sums are added in a fixed tree.
// Deterministic: the same schedule always gives the same bits.
__global__ void __launch_bounds__(128) k_accum_part(const int4 *__restrict__ chunk, const int32_t *__restrict__ order,
                                                    const uint32_t *__restrict__ mass, const float *__restrict__ val,
                                                    int32_t R, int32_t ore_off, const double *__restrict__ grade,
                                                    int32_t S, int64_t *__restrict__ p_ore, double *__restrict__ p_met,
                                                    int64_t *__restrict__ p_mass) {
    const int4 c = chunk[blockIdx.x];  // (period, begin, end, 0)
    int64_t mt = 0;                    // the chunk's mined tonnage (thread 0, in its s = 0 pass)
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        int64_t o = 0;
        double g = 0.0;
        for (int32_t k0 = c.y; k0 < c.z; k0 += 8) {
            int32_t b[8];
            uint32_t mb[8], ob[8];
            double gb[8];
#pragma unroll
            for (int u = 0; u < 8; u++) b[u] = k0 + u < c.z ? __ldg(order + k0 + u) : -1;
#pragma unroll
            for (int u = 0; u < 8; u++) {
                mb[u] = ob[u] = 0u;
                gb[u] = 0.0;
                if (b[u] >= 0) {
                    mb[u] = __ldg(mass + b[u]);
                    ob[u] = ore_bit(val, R, ore_off, b[u], s);
                    gb[u] = __ldg(grade + (int64_t)b[u] * S + s);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                if (s == 0) mt += mb[u];  // 0 past the chunk's end
                if (ob[u]) {
                    o += mb[u];
                    g = __dadd_rn(g, __dmul_rn((double)mb[u], gb[u]));
                }
            }
        }
        p_ore[(int64_t)blockIdx.x * S + s] = o;
        p_met[(int64_t)blockIdx.x * S + s] = g;
    }
    if (threadIdx.x == 0) p_mass[blockIdx.x] = mt;
}

__global__ void __launch_bounds__(256) k_accum_reduce(const int32_t *__restrict__ cbase,
                                                      const int64_t *__restrict__ p_ore,
                                                      const double *__restrict__ p_met,
                                                      const int64_t *__restrict__ p_mass, int32_t S,
                                                      int64_t *__restrict__ minedT, int64_t *__restrict__ oreT,
                                                      double *__restrict__ metal) {
    __shared__ int64_t s_o[8][32];
    __shared__ double s_g[8][32];
    const int t = blockIdx.x;
    const int j = threadIdx.x & 31, u = threadIdx.x >> 5;  // scenario lane, chunk subset (warp)
    const int s = blockIdx.y * 32 + j;
    const int32_t c0 = cbase[t], c1 = cbase[t + 1];
    // warp u: chunks c0 + u, c0 + u + 8, ... in chunk order, four loads in flight
    int64_t o = 0;
    double g = 0.0;
    if (s < S) {
        for (int32_t c = c0 + u; c < c1; c += 32) {
            int64_t ob[4];
            double gb[4];
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const int32_t cc = c + 8 * v;
                ob[v] = cc < c1 ? p_ore[(int64_t)cc * S + s] : 0;
                gb[v] = cc < c1 ? p_met[(int64_t)cc * S + s] : 0.0;
            }
#pragma unroll
            for (int v = 0; v < 4; v++)
                if (c + 8 * v < c1) {
                    o += ob[v];
                    g = __dadd_rn(g, gb[v]);
                }
        }
    }
    s_o[u][j] = o;
    s_g[u][j] = g;
    // the period's mined tonnage: warp 0 of the first scenario group (exact integers)
    int64_t mt = 0;
    if (blockIdx.y == 0 && u == 0) {
        for (int32_t c = c0 + j; c < c1; c += 32) mt += p_mass[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) mt += __shfl_down_sync(0xffffffffu, mt, off);
    }
    __syncthreads();
    if (u == 0 && s < S) {
        // the eight subsets' sums in a fixed tree
        const double a0 = __dadd_rn(s_g[0][j], s_g[1][j]), a1 = __dadd_rn(s_g[2][j], s_g[3][j]);
        const double a2 = __dadd_rn(s_g[4][j], s_g[5][j]), a3 = __dadd_rn(s_g[6][j], s_g[7][j]);
        int64_t ot = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) ot += s_o[k][j];
        oreT[(int64_t)t * S + s] = ot;
        metal[(int64_t)t * S + s] = __dadd_rn(__dadd_rn(a0, a1), __dadd_rn(a2, a3));
    }
    if (blockIdx.y == 0 && threadIdx.x == 0) minedT[t] = mt;
}

__global__ void k_tables(int32_t S, int32_t S_pad, int32_t T, const int64_t *__restrict__ oreT,
                         const uint64_t *__restrict__ target, const double *__restrict__ disc, int64_t m, double a,
                         double e, float *__restrict__ tab, float4 *__restrict__ tabc) {
    int t = blockIdx.x;
    for (int s = threadIdx.x; s < S_pad; s += blockDim.x) table_entry(t, s, S, S_pad, T, oreT, target, disc, m, a, e, tab);
    if (threadIdx.x == 0) tabc[t] = table_consts(t, T, disc, m, a, e);
}

// ctab[a][b][s] = Pout[a][s] + Pin[b][s], the FP32 sum the evaluator would form.
__global__ void k_ctab(int32_t S_pad, int32_t T, const float *__restrict__ tab, float *__restrict__ ctab) {
    const int T1 = T + 1;
    const int a = blockIdx.x / T1, b = blockIdx.x % T1;
    const float *po = tab + (int64_t)a * S_pad;
    const float *pi = tab + (int64_t)T1 * S_pad + (int64_t)b * S_pad;
    float *dst = ctab + (int64_t)blockIdx.x * S_pad;
    for (int s = threadIdx.x; s < S_pad; s += blockDim.x) dst[s] = po[s] + pi[s];
}

// contrib[t][s] for every period, and NPV_s = their sum in period order.
__global__ void k_npv(int32_t S, int32_t T, const double *__restrict__ disc, const double *__restrict__ metal,
                      const int64_t *__restrict__ oreT, const int64_t *__restrict__ minedT,
                      const uint64_t *__restrict__ target, double pr, double pc, double mc, double a, double e,
                      const double *__restrict__ sig, double *__restrict__ contrib, double *__restrict__ npv) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    double acc = 0.0;
    for (int t = 0; t < T; t++) {
        double c = contrib_of(t, s, S, disc, metal, oreT, minedT, target, pr, pc, mc, a, e, sig);
        contrib[(int64_t)t * S + s] = c;
        acc = __dadd_rn(acc, c);
    }
    npv[s] = acc;
}

// FP32 shadow accumulators from the current FP64 state: metal rounded to FP32,
// the period contributions recomputed in FP32 from it and the exact integer
// tonnages, NPV_s their FP32 sum in period order.
__global__ void k_shadow_init(int32_t S, int32_t T, const double *__restrict__ disc, const double *__restrict__ metal,
                              const int64_t *__restrict__ oreT, const int64_t *__restrict__ minedT,
                              const uint64_t *__restrict__ target, double pr, double pc, double mc, double a, double e,
                              const double *__restrict__ sig, float *__restrict__ shadow) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    float *metal32 = shadow, *contrib32 = shadow + (size_t)T * S, *npv32 = contrib32 + (size_t)T * S;
    float acc = 0.0f;
    for (int t = 0; t < T; t++) {
        const size_t i = (size_t)t * S + s;
        const float mf = (float)metal[i];
        const float c = contrib_val_f32(oreT[i], mf, minedT[t], (int64_t)target[t], disc[t], pr, pc, mc, a, e,
                                        sig ? sig[i] : 1.0);
        metal32[i] = mf;
        contrib32[i] = c;
        acc += c;
    }
    npv32[s] = acc;
}

static mm_status shadow_init(mm_model *m) {
    if (!m->shadow32) return MM_OK;
    k_shadow_init<<<(m->S + 127) / 128, 128, 0, m->stream>>>(m->S, m->T, m->disc, m->metal, m->oreT, m->minedT,
                                                             m->target, m->price * m->recovery, m->proc_cost,
                                                             m->mining_cost, m->shortfall_pen, m->excess_pen,
                                                             m->sig, m->shadow32);
    return check_launch("k_shadow_init");
}

// Apply kernel: the move comes either by value (from_dev = 0) or as
// moves[idx[0]] when *count > 0 (from_dev = 1; an index outside the batch is a
// bad move).
__global__ void __launch_bounds__(1024) k_apply(ApplyArgs A, int2 mv_val, const int2 *moves, int64_t n_moves, const int32_t *idx,
                        const int32_t *count, int from_dev) {
    __shared__ __align__(16) float s_tab[kApplyTabMax];
    int2 mv = mv_val;
    int have = 1;
    if (from_dev) {
        have = *count > 0;
        if (have) {
            const int32_t j = idx[0];
            if (j >= 0 && (int64_t)j < n_moves) {
                mv = moves[j];
            } else {
                mv = make_int2(-1, -1);  // decodes as a bad move
                if (threadIdx.x == 0) atomicOr(A.status, kStBadMove);
            }
        }
    }
    apply_block(A, mv, have, s_tab);
}

// The FP64 part of the move a fused step applied structurally (*pending, if
// still due): metal, net cash and NPV_s, then the record is cleared.
__global__ void __launch_bounds__(1024) k_apply_pending(ApplyArgs A, int4 *pending) {
    const int4 p = *pending;
    if (p.w) apply_money(A, p, threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) pending->w = 0;
}

// NPV mean and population std over scenarios of the current schedule (FP64,
// two passes) into the model's apply result; one CTA.
__global__ void k_npv_stats(const double *__restrict__ npv, int32_t S, ApplyResult *res) {
    __shared__ double red[32];
    __shared__ double s_mean;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double x = 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) x = __dadd_rn(x, npv[s]);
    x = warp_sum_f64(x);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    if (warp == 0) {
        double y = lane < nw ? red[lane] : 0.0;
        y = warp_sum_f64(y);
        if (lane == 0) s_mean = y / (double)S;
    }
    __syncthreads();
    const double mean = s_mean;
    double q = 0.0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double d = __dsub_rn(npv[s], mean);
        q = __fma_rn(d, d, q);
    }
    q = warp_sum_f64(q);
    __syncthreads();
    if (lane == 0) red[warp] = q;
    __syncthreads();
    if (warp == 0) {
        double y = lane < nw ? red[lane] : 0.0;
        y = warp_sum_f64(y);
        if (lane == 0) {
            res->mean = mean;
            res->std = sqrt(y / (double)S);
        }
    }
}

static mm_status npv_stats_launch(mm_model *m) {
    k_npv_stats<<<1, 256, 0, m->stream>>>(m->npv, m->S, m->apply_res);
    return check_launch("k_npv_stats");
}

// ------------------------------------------------------------------ host

mm_status rebuild_tables(mm_model *m) {
    if (!m->uniform_mass) return MM_OK;
    k_tables<<<m->T + 1, 128, 0, m->stream>>>(m->S, m->S_pad, m->T, m->oreT, m->target, m->disc, (int64_t)m->m_uniform,
                                              m->shortfall_pen, m->excess_pen, m->tab,
                                              reinterpret_cast<float4 *>(m->tabc));
    mm_status st = check_launch("k_tables");
    if (st != MM_OK || !m->ctab) return st;
    k_ctab<<<(m->T + 1) * (m->T + 1), 128, 0, m->stream>>>(m->S_pad, m->T, m->tab, m->ctab);
    return check_launch("k_ctab");
}

ApplyArgs apply_args(mm_model *m) {
    ApplyArgs A;
    A.tp = topo_of(m);
    A.S = m->S; A.S_pad = m->S_pad; A.W = m->W; A.T = m->T; A.R = m->R; A.ore_off = m->ore_off;
    A.m_uniform = m->m_uniform; A.uniform = m->uniform_mass;
    A.mass = m->mass; A.val = m->val; A.grade = m->grade; A.blk = m->blk;
    A.minedT = m->minedT; A.oreT = m->oreT; A.metal = m->metal; A.npv = m->npv; A.contrib = m->contrib;
    A.tab = m->tab;
    A.tabc = reinterpret_cast<const float4 *>(m->tabc);
    A.ctab = m->ctab;
    A.disc = m->disc; A.sig = m->sig; A.cap = m->cap; A.target = m->target;
    A.pr = m->price * m->recovery; A.pc = m->proc_cost; A.mc = m->mining_cost;
    A.a = m->shortfall_pen; A.e = m->excess_pen;
    A.res = m->apply_res;
    A.status = m->status;
    A.metal32 = m->shadow32;
    A.contrib32 = m->shadow32 ? m->shadow32 + (size_t)m->T * m->S : nullptr;
    A.npv32 = m->shadow32 ? m->shadow32 + 2 * (size_t)m->T * m->S : nullptr;
    return A;
}

static int apply_threads(const mm_model *m);

mm_status settle_money(mm_model *m, cudaStream_t stream) {
    if (!m->money_due) return MM_OK;
    k_apply_pending<<<1, apply_threads(m), 0, stream ? stream : m->stream>>>(apply_args(m), m->pending);
    mm_status st = check_launch("k_apply_pending");
    if (st == MM_OK) m->money_due = 0;
    return st;
}

static int apply_threads(const mm_model *m) {
    int t = ((m->S + 31) / 32) * 32;
    if (t < 64) t = 64;
    if (m->ctab && t < 512) t = 512;  // the period-pair rows are rebuilt by the whole CTA
    if (t > 1024) t = 1024;
    return t;
}

}  // namespace mm

using namespace mm;

template <typename T>
static mm_status dalloc(T **p, size_t count, const char *what) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    // host-side fault injection for tests: with MM_ALLOC_CAP_BYTES set, an
    // allocation larger than it fails as out of memory before any CUDA call
    if (const char *cap = std::getenv("MM_ALLOC_CAP_BYTES")) {
        if (*cap && bytes > (size_t)std::strtoull(cap, nullptr, 10)) {
            *p = nullptr;
            return set_error(MM_ERR_OOM, "%s: %zu bytes exceed MM_ALLOC_CAP_BYTES", what, bytes);
        }
    }
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_status(e, what);
    }
    return MM_OK;
}

extern "C" {

const char *mm_last_error(void) { return g_err; }

void mm_model_destroy(mm_model *m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->mass); cudaFree(m->grade); cudaFree(m->val); cudaFree(m->blk);
    cudaFree(m->pred_ptr); cudaFree(m->pred_idx); cudaFree(m->succ_ptr); cudaFree(m->succ_idx);
    cudaFree(m->order); cudaFree(m->porder);
    cudaFree(m->accum_chunk); cudaFree(m->accum_cbase); cudaFree(m->accum_ore); cudaFree(m->accum_met);
    cudaFree(m->accum_mass);
    cudaFree(m->minedT); cudaFree(m->oreT); cudaFree(m->metal); cudaFree(m->npv); cudaFree(m->contrib);
    cudaFree(m->tab);
    cudaFree(m->ctab);
    cudaFree(m->sig); cudaFree(m->dwt);
    cudaFree(m->ddt); cudaFree(m->disc); cudaFree(m->cap); cudaFree(m->target); cudaFree(m->status);
    cudaFree(m->apply_res);
    cudaFree(m->step_cta);
    cudaFree(m->step_grp);
    cudaFree(m->step_cinf);
    cudaFree(m->step_ginf);
    cudaFree(m->step_tick);
    cudaFree(m->pending);
    cudaFree(m->tabc);
    cudaFree(m->relax_scratch);
    cudaFree(m->relax_coef);
    cudaFree(m->relax_tick);
    cudaFree(m->shadow32);
    if (m->apply_res_host) cudaFreeHost(m->apply_res_host);
    if (m->status_host) cudaFreeHost(m->status_host);
    topk_scratch_free(m->topk);
    delete m;
}

mm_status mm_model_create(const mm_model_desc *d, mm_model **out) {
    g_err[0] = 0;
    if (!d || !out) return set_error(MM_ERR_INVALID_ARG, "mm_model_create: NULL argument");
    *out = nullptr;
    const int32_t B = d->n_blocks, S = d->n_scenarios, T = d->n_periods;
    if (B <= 0 || S <= 0 || T <= 0) return set_error(MM_ERR_INVALID_ARG, "B, S and T must be positive");
    if (S > kMaxS) return set_error(MM_ERR_INVALID_ARG, "S = %d exceeds the limit %d", S, kMaxS);
    if (T > kMaxT) return set_error(MM_ERR_INVALID_ARG, "T = %d exceeds the limit %d", T, kMaxT);
    if (!d->mass_t || !d->grade || !d->cap_t || !d->mill_target_t)
        return set_error(MM_ERR_INVALID_ARG, "mass, grade, capacity and mill target are required");
    bool grid = d->nx > 0 || d->ny > 0 || d->nz > 0;
    if (grid) {
        if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || (int64_t)d->nx * d->ny * d->nz != B)
            return set_error(MM_ERR_INVALID_ARG, "grid %d x %d x %d does not hold %d blocks", d->nx, d->ny, d->nz, B);
    } else if (!d->pred_ptr || !d->pred_idx) {
        return set_error(MM_ERR_INVALID_ARG, "either a grid or a predecessor CSR is required");
    }
    const double econ[] = {d->price, d->recovery, d->mining_cost, d->proc_cost, d->shortfall_pen, d->excess_pen,
                           d->discount_rate, d->lambda};
    for (double v : econ)
        if (!std::isfinite(v)) return set_error(MM_ERR_INVALID_ARG, "economic parameters must be finite");
    if (d->discount_rate <= -1.0) return set_error(MM_ERR_INVALID_ARG, "discount rate must exceed -1");
    uint64_t total = 0;
    for (int32_t b = 0; b < B; b++) {
        if (d->mass_t[b] == 0) return set_error(MM_ERR_INVALID_ARG, "block %d has zero mass", b);
        total += d->mass_t[b];
    }
    if (total >= (1ull << 62)) return set_error(MM_ERR_OVERFLOW, "total block mass exceeds 2^62 t");
    for (int32_t t = 0; t < T; t++)
        if (d->cap_t[t] >= (1ull << 62) || d->mill_target_t[t] >= (1ull << 62))
            return set_error(MM_ERR_OVERFLOW, "capacity or mill target of period %d exceeds 2^62 t", t);
    for (int64_t i = 0; i < (int64_t)B * S; i++)
        if (!std::isfinite(d->grade[i]) || d->grade[i] < 0.0)
            return set_error(MM_ERR_INVALID_ARG, "grade[%lld] is negative or not finite", (long long)i);
    if (d->sigma)
        for (int64_t i = 0; i < (int64_t)T * S; i++)
            if (!std::isfinite(d->sigma[i]) || d->sigma[i] < 0.0)
                return set_error(MM_ERR_INVALID_ARG, "sigma[%lld] is negative or not finite", (long long)i);
    std::vector<int32_t> sptr, sidx;
    if (!grid) {
        if (d->pred_ptr[0] != 0) return set_error(MM_ERR_INVALID_ARG, "pred_ptr[0] must be 0");
        for (int32_t b = 0; b < B; b++)
            if (d->pred_ptr[b + 1] < d->pred_ptr[b]) return set_error(MM_ERR_INVALID_ARG, "pred_ptr is not monotone");
        int32_t E = d->pred_ptr[B];
        for (int32_t k = 0; k < E; k++)
            if (d->pred_idx[k] < 0 || d->pred_idx[k] >= B)
                return set_error(MM_ERR_INVALID_ARG, "pred_idx[%d] out of range", k);
        for (int32_t b = 0; b < B; b++)
            for (int32_t k = d->pred_ptr[b]; k < d->pred_ptr[b + 1]; k++)
                if (d->pred_idx[k] == b) return set_error(MM_ERR_INVALID_ARG, "block %d is its own predecessor", b);
        sptr.assign(B + 1, 0);
        for (int32_t k = 0; k < E; k++) sptr[d->pred_idx[k] + 1]++;
        for (int32_t b = 0; b < B; b++) sptr[b + 1] += sptr[b];
        sidx.assign(E > 0 ? E : 1, 0);
        std::vector<int32_t> fill(sptr.begin(), sptr.end() - 1);
        for (int32_t b = 0; b < B; b++)
            for (int32_t k = d->pred_ptr[b]; k < d->pred_ptr[b + 1]; k++) sidx[fill[d->pred_idx[k]]++] = b;
    }

    mm_model *m = new mm_model();
    m->B = B; m->S = S; m->T = T;
    // test-only: the bulk-copy evaluator's stages wait for bytes that never
    // come (every copy it issues still lands), so its bounded wait runs out
    if (const char *st = std::getenv("MM_TEST_STALL_BULK_WAIT")) m->test_stall = (*st && *st != '0') ? 1 : 0;
    if (const char *st = std::getenv("MM_TEST_STALL_RELAXED")) m->test_stall_relax = (*st && *st != '0') ? 1 : 0;
    m->S_pad = (S + 7) / 8 * 8;
    m->W = (S + 31) / 32;
    m->ore_off = 4 * ((S + 3) / 4);
    m->R = (m->ore_off + m->W + 7) / 8 * 8;
    m->nx = grid ? d->nx : 0; m->ny = grid ? d->ny : 0; m->nz = grid ? d->nz : 0;
    m->price = d->price; m->recovery = d->recovery; m->mining_cost = d->mining_cost; m->proc_cost = d->proc_cost;
    m->shortfall_pen = d->shortfall_pen; m->excess_pen = d->excess_pen; m->discount_rate = d->discount_rate;
    m->lambda = d->lambda;
    m->stream = (cudaStream_t)d->cuda_stream;
    m->uniform_mass = 1;
    m->m_uniform = d->mass_t[0];
    for (int32_t b = 1; b < B; b++)
        if (d->mass_t[b] != m->m_uniform) { m->uniform_mass = 0; break; }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
    {
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess && l2 > 0) m->l2_bytes = (size_t)l2;
    }
    cudaDeviceGetAttribute(&m->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);

    m->h_disc.resize(T + 1);
    for (int t = 0; t < T; t++) m->h_disc[t] = std::pow(1.0 + d->discount_rate, -(double)t);
    m->h_disc[T] = 0.0;
    m->h_cap.assign(d->cap_t, d->cap_t + T);
    m->h_target.assign(d->mill_target_t, d->mill_target_t + T);

    mm_status st = MM_OK;
#define ALLOC(ptr, n) \
    if (st == MM_OK) st = dalloc(&m->ptr, (size_t)(n), "allocate " #ptr)
    ALLOC(mass, B);
    ALLOC(grade, (int64_t)B * S);
    ALLOC(val, (int64_t)(B + 1) * m->R);
    ALLOC(blk, B);
    ALLOC(order, B);
    ALLOC(porder, T + 2);
    // schedule_set's chunked sums: about 1,600 chunks (at least 32 blocks each)
    m->accum_chunk_len = std::max<int32_t>(32, (B + 1599) / 1600);
    m->accum_max_chunks = (B + m->accum_chunk_len - 1) / m->accum_chunk_len + T;
    ALLOC(accum_chunk, m->accum_max_chunks);
    ALLOC(accum_cbase, T + 1);
    ALLOC(accum_ore, (size_t)m->accum_max_chunks * S);
    ALLOC(accum_met, (size_t)m->accum_max_chunks * S);
    ALLOC(accum_mass, m->accum_max_chunks);
    ALLOC(minedT, T + 1);
    ALLOC(oreT, (int64_t)(T + 1) * S);
    ALLOC(metal, (int64_t)T * S);
    ALLOC(npv, S);
    ALLOC(contrib, (int64_t)T * S);
    ALLOC(tab, (int64_t)2 * (T + 1) * m->S_pad);
    if (T <= kCtabMaxT && m->uniform_mass) ALLOC(ctab, (int64_t)(T + 1) * (T + 1) * m->S_pad);
    ALLOC(ddt, (int64_t)(T + 1) * (T + 1));
    if (d->sigma) {
        ALLOC(sig, (int64_t)T * S);
        ALLOC(dwt, (int64_t)(T + 1) * (T + 1) * m->S_pad);
    }
    ALLOC(disc, T + 1);
    ALLOC(cap, T + 1);
    ALLOC(target, T + 1);
    ALLOC(status, 1);
    ALLOC(apply_res, 1);
    m->step_max_ctas = m->num_sms * 8;  // 256-thread CTAs: at most 8 resident per SM
    ALLOC(step_cta, (size_t)m->step_max_ctas * 32);
    ALLOC(step_grp, (size_t)m->step_max_ctas * 32);
    ALLOC(step_cinf, (size_t)m->step_max_ctas);
    ALLOC(step_ginf, (size_t)m->step_max_ctas);
    ALLOC(step_tick, (size_t)m->step_max_ctas + 1);
    ALLOC(pending, 1);
    ALLOC(tabc, (int64_t)4 * (T + 1));
    ALLOC(relax_tick, 1);
    if (!grid) {
        ALLOC(pred_ptr, B + 1);
        ALLOC(pred_idx, d->pred_ptr[B] > 0 ? d->pred_ptr[B] : 1);
        ALLOC(succ_ptr, B + 1);
        ALLOC(succ_idx, sidx.size());
    }
#undef ALLOC
    if (st == MM_OK && cudaMallocHost((void **)&m->apply_res_host, sizeof(ApplyResult)) != cudaSuccess)
        st = set_error(MM_ERR_OOM, "pinned host allocation failed");
    if (st == MM_OK && cudaMallocHost((void **)&m->status_host, sizeof(uint32_t)) != cudaSuccess)
        st = set_error(MM_ERR_OOM, "pinned host allocation failed");
    if (st != MM_OK) {
        mm_model_destroy(m);
        return st;
    }
    auto fail = [&](mm_status s) {
        mm_model_destroy(m);
        return s;
    };
    cudaStream_t s = m->stream;
#define TRY(expr, what)                                   \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return fail(cuda_status(e_, what)); \
    } while (0)
    TRY(cudaMemcpyAsync(m->mass, d->mass_t, sizeof(uint32_t) * B, cudaMemcpyHostToDevice, s), "copy mass");
    TRY(cudaMemcpyAsync(m->grade, d->grade, sizeof(double) * (size_t)B * S, cudaMemcpyHostToDevice, s), "copy grade");
    std::vector<uint64_t> capx(T + 1), tgtx(T + 1);
    for (int t = 0; t < T; t++) capx[t] = d->cap_t[t], tgtx[t] = d->mill_target_t[t];
    capx[T] = std::numeric_limits<uint64_t>::max();
    tgtx[T] = 0;
    std::vector<float> ddt((size_t)(T + 1) * (T + 1));
    for (int t = 0; t <= T; t++)
        for (int u = 0; u <= T; u++) ddt[(size_t)t * (T + 1) + u] = (float)(m->h_disc[u] - m->h_disc[t]);
    TRY(cudaMemcpyAsync(m->cap, capx.data(), sizeof(uint64_t) * (T + 1), cudaMemcpyHostToDevice, s), "copy cap");
    TRY(cudaMemcpyAsync(m->target, tgtx.data(), sizeof(uint64_t) * (T + 1), cudaMemcpyHostToDevice, s), "copy target");
    TRY(cudaMemcpyAsync(m->disc, m->h_disc.data(), sizeof(double) * (T + 1), cudaMemcpyHostToDevice, s), "copy disc");
    TRY(cudaMemcpyAsync(m->ddt, ddt.data(), sizeof(float) * ddt.size(), cudaMemcpyHostToDevice, s), "copy ddt");
    std::vector<float> dwt;
    if (d->sigma) {
        // weighted discount W[t][s] = sigma(s,t) d_t (W[T] = 0, unmined) and
        // its period-pair differences, each formed in FP64 and rounded once
        const int T1 = T + 1, Sp = m->S_pad;
        std::vector<double> w((size_t)T1 * S, 0.0);
        for (int t = 0; t < T; t++)
            for (int sc = 0; sc < S; sc++) w[(size_t)t * S + sc] = d->sigma[(size_t)t * S + sc] * m->h_disc[t];
        dwt.assign((size_t)T1 * T1 * Sp, 0.0f);
        for (int a = 0; a <= T; a++)
            for (int b = 0; b <= T; b++)
                for (int sc = 0; sc < S; sc++)
                    dwt[((size_t)a * T1 + b) * Sp + sc] = (float)(w[(size_t)b * S + sc] - w[(size_t)a * S + sc]);
        TRY(cudaMemcpyAsync(m->sig, d->sigma, sizeof(double) * (size_t)T * S, cudaMemcpyHostToDevice, s), "copy sigma");
        TRY(cudaMemcpyAsync(m->dwt, dwt.data(), sizeof(float) * dwt.size(), cudaMemcpyHostToDevice, s), "copy dwt");
    }
    TRY(cudaMemsetAsync(m->status, 0, sizeof(uint32_t), s), "clear status");
    TRY(cudaMemsetAsync(m->val, 0, sizeof(float) * (size_t)(B + 1) * m->R, s), "clear rows");
    TRY(cudaMemsetAsync(m->oreT, 0, sizeof(int64_t) * (size_t)(T + 1) * S, s), "clear oreT");
    TRY(cudaMemsetAsync(m->minedT, 0, sizeof(int64_t) * (T + 1), s), "clear minedT");
    TRY(cudaMemsetAsync(m->apply_res, 0, sizeof(ApplyResult), s), "clear apply result");
    TRY(cudaMemsetAsync(m->step_tick, 0, sizeof(uint32_t) * ((size_t)m->step_max_ctas + 1), s), "clear step tickets");
    TRY(cudaMemsetAsync(m->pending, 0, sizeof(int4), s), "clear the pending apply");
    TRY(cudaMemsetAsync(m->relax_tick, 0, sizeof(uint32_t), s), "clear relaxed ticket");
    if (!grid) {
        TRY(cudaMemcpyAsync(m->pred_ptr, d->pred_ptr, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s), "copy CSR");
        if (d->pred_ptr[B] > 0)
            TRY(cudaMemcpyAsync(m->pred_idx, d->pred_idx, sizeof(int32_t) * d->pred_ptr[B], cudaMemcpyHostToDevice, s),
                "copy CSR");
        TRY(cudaMemcpyAsync(m->succ_ptr, sptr.data(), sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s), "copy CSR");
        TRY(cudaMemcpyAsync(m->succ_idx, sidx.data(), sizeof(int32_t) * sidx.size(), cudaMemcpyHostToDevice, s),
            "copy CSR");
    }
    int64_t nthreads = (int64_t)B * m->W;
    k_classify<<<(unsigned)((nthreads + 255) / 256), 256, 0, s>>>(m->grade, m->mass, B, S, m->R, m->ore_off, m->W,
                                                                  m->price, m->recovery, m->proc_cost, m->mining_cost,
                                                                  m->sig ? 1 : 0, m->val);
    mm_status ls = check_launch("k_classify");
    if (ls != MM_OK) return fail(ls);
    TRY(cudaStreamSynchronize(s), "synchronize after create");
#undef TRY
    *out = m;
    return MM_OK;
}

mm_status mm_set_stream(mm_model *m, void *stream) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    m->stream = (cudaStream_t)stream;
    return MM_OK;
}

mm_status mm_model_info(const mm_model *m, int32_t *B, int32_t *S, int32_t *T, int32_t *s_pad) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (B) *B = m->B;
    if (S) *S = m->S;
    if (T) *T = m->T;
    if (s_pad) *s_pad = m->R;
    return MM_OK;
}

mm_status mm_schedule_set(mm_model *m, const uint8_t *period, int *base_feasible_out) {
    if (!m || !period) return set_error(MM_ERR_INVALID_ARG, "mm_schedule_set: NULL argument");
    const int32_t B = m->B, T = m->T, S = m->S;
    std::vector<int32_t> cnt(T + 2, 0);
    for (int32_t b = 0; b < B; b++) {
        if (period[b] > T) return set_error(MM_ERR_INVALID_ARG, "period[%d] = %d exceeds T = %d", b, period[b], T);
        cnt[period[b] + 1]++;
    }
    for (int t = 0; t <= T; t++) cnt[t + 1] += cnt[t];
    std::vector<int32_t> order(B), fill(cnt.begin(), cnt.end() - 1);
    for (int32_t b = 0; b < B; b++) order[fill[period[b]]++] = b;
    // chunks of each mined period's blocks (period T, unmined, is not summed)
    std::vector<int4> chunks;
    std::vector<int32_t> cbase(T + 1, 0);
    const int32_t CL = m->accum_chunk_len;
    for (int t = 0; t < T; t++) {
        cbase[t] = (int32_t)chunks.size();
        for (int32_t k = cnt[t]; k < cnt[t + 1]; k += CL) chunks.push_back(make_int4(t, k, std::min(k + CL, cnt[t + 1]), 0));
    }
    cbase[T] = (int32_t)chunks.size();
    cudaStream_t s = m->stream;
    uint8_t *d_period = nullptr;
    mm_status st = dalloc(&d_period, B, "allocate period staging");
    if (st != MM_OK) return st;
    auto done = [&](mm_status r) {
        cudaStreamSynchronize(s);
        cudaFree(d_period);
        return r;
    };
#define TRY(expr, what)                                   \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return done(cuda_status(e_, what)); \
    } while (0)
    // every total is rebuilt from the new schedule: an FP64 update still due is void
    TRY(cudaMemsetAsync(m->pending, 0, sizeof(int4), s), "clear the pending apply");
    m->money_due = 0;
    TRY(cudaMemcpyAsync(d_period, period, B, cudaMemcpyHostToDevice, s), "copy schedule");
    TRY(cudaMemcpyAsync(m->order, order.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s), "copy order");
    TRY(cudaMemcpyAsync(m->porder, cnt.data(), sizeof(int32_t) * (T + 2), cudaMemcpyHostToDevice, s), "copy order");
    Topo tp = topo_of(m);
    k_blk_build<<<(B + 255) / 256, 256, 0, s>>>(tp, d_period, m->blk);
    if ((st = check_launch("k_blk_build")) != MM_OK) return done(st);
    TRY(cudaMemsetAsync(m->oreT, 0, sizeof(int64_t) * (size_t)(T + 1) * S, s), "clear oreT");
    TRY(cudaMemsetAsync(m->minedT, 0, sizeof(int64_t) * (T + 1), s), "clear minedT");
    if (!chunks.empty()) {
        TRY(cudaMemcpyAsync(m->accum_chunk, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice, s),
            "copy chunk table");
        TRY(cudaMemcpyAsync(m->accum_cbase, cbase.data(), sizeof(int32_t) * (T + 1), cudaMemcpyHostToDevice, s),
            "copy chunk offsets");
        k_accum_part<<<(unsigned)chunks.size(), 128, 0, s>>>(m->accum_chunk, m->order, m->mass, m->val, m->R,
                                                             m->ore_off, m->grade, S, m->accum_ore, m->accum_met,
                                                             m->accum_mass);
        if ((st = check_launch("k_accum_part")) != MM_OK) return done(st);
        k_accum_reduce<<<dim3(T, (S + 31) / 32), 256, 0, s>>>(m->accum_cbase, m->accum_ore, m->accum_met,
                                                                m->accum_mass, S, m->minedT, m->oreT, m->metal);
        if ((st = check_launch("k_accum_reduce")) != MM_OK) return done(st);
    } else {
        TRY(cudaMemsetAsync(m->metal, 0, sizeof(double) * (size_t)T * S, s), "clear metal");
    }
    if ((st = rebuild_tables(m)) != MM_OK) return done(st);
    k_npv<<<(S + 127) / 128, 128, 0, s>>>(S, T, m->disc, m->metal, m->oreT, m->minedT, m->target,
                                           m->price * m->recovery, m->proc_cost, m->mining_cost, m->shortfall_pen,
                                           m->excess_pen, m->sig, m->contrib, m->npv);
    if ((st = check_launch("k_npv")) != MM_OK) return done(st);
    if ((st = shadow_init(m)) != MM_OK) return done(st);
    // base feasibility: arcs (device) + capacity (host, from minedT)
    uint32_t *d_bad = m->status_host ? nullptr : nullptr;
    TRY(cudaMemsetAsync(m->apply_res, 0, sizeof(ApplyResult), s), "clear apply result");
    d_bad = (uint32_t *)&m->apply_res->status;  // reuse as a scratch word
    k_base_arcs<<<(B + 255) / 256, 256, 0, s>>>(B, m->blk, d_bad);
    if ((st = check_launch("k_base_arcs")) != MM_OK) return done(st);
    std::vector<int64_t> mined(T + 1);
    TRY(cudaMemcpyAsync(mined.data(), m->minedT, sizeof(int64_t) * (T + 1), cudaMemcpyDeviceToHost, s), "read minedT");
    TRY(cudaMemcpyAsync(m->apply_res_host, m->apply_res, sizeof(ApplyResult), cudaMemcpyDeviceToHost, s),
        "read feasibility");
    TRY(cudaStreamSynchronize(s), "synchronize");
    int feas = m->apply_res_host->status == 0;
    for (int t = 0; t < T; t++)
        if ((uint64_t)mined[t] > m->h_cap[t]) feas = 0;
    TRY(cudaMemsetAsync(m->apply_res, 0, sizeof(ApplyResult), s), "clear apply result");
#undef TRY
    if (base_feasible_out) *base_feasible_out = feas;
    m->has_schedule = 1;
    return done(MM_OK);
}

mm_status mm_schedule_get(mm_model *m, uint8_t *period) {
    if (!m || !period) return set_error(MM_ERR_INVALID_ARG, "mm_schedule_get: NULL argument");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    std::vector<uint32_t> w(m->B);
    MM_CUDA_TRY(cudaMemcpyAsync(w.data(), m->blk, sizeof(uint32_t) * m->B, cudaMemcpyDeviceToHost, m->stream),
                "read schedule");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    for (int32_t b = 0; b < m->B; b++) period[b] = (uint8_t)blk_period(w[b]);
    return read_sticky(m);
}

mm_status mm_apply_move(mm_model *m, mm_move mv, double *mean, double *sd) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    mm_status ss = settle_money(m);
    if (ss != MM_OK) return ss;
    ApplyArgs A = apply_args(m);
    k_apply<<<1, apply_threads(m), 0, m->stream>>>(A, make_int2(mv.b1, mv.arg), nullptr, 0, nullptr, nullptr, 0);
    mm_status st = check_launch("k_apply");
    if (st != MM_OK) return st;
    if ((st = npv_stats_launch(m)) != MM_OK) return st;
    MM_CUDA_TRY(cudaMemcpyAsync(m->apply_res_host, m->apply_res, sizeof(ApplyResult), cudaMemcpyDeviceToHost, m->stream),
                "read apply result");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    ApplyResult r = *m->apply_res_host;
    mm_status sticky = read_sticky(m);
    if (r.status == MM_ERR_BAD_MOVE) return set_error(MM_ERR_BAD_MOVE, "move (%d, %d) is out of range", mv.b1, mv.arg);
    if (r.status == MM_ERR_INFEASIBLE) return set_error(MM_ERR_INFEASIBLE, "move (%d, %d) is infeasible", mv.b1, mv.arg);
    if (mean) *mean = r.mean;
    if (sd) *sd = r.std;
    return sticky;
}

mm_status mm_apply_best(mm_model *m, const mm_move *moves, int64_t n, const int32_t *idx, const int32_t *count) {
    if (!m || (!moves && n > 0) || !idx || !count) return set_error(MM_ERR_INVALID_ARG, "mm_apply_best: NULL argument");
    if (n < 0) return set_error(MM_ERR_INVALID_ARG, "negative move count");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    mm_status ss = settle_money(m);
    if (ss != MM_OK) return ss;
    ApplyArgs A = apply_args(m);
    k_apply<<<1, apply_threads(m), 0, m->stream>>>(A, make_int2(0, 0), (const int2 *)moves, n, idx, count, 1);
    return check_launch("k_apply");
}

mm_status mm_set_fp32_shadow(mm_model *m, int32_t enable) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    mm_status ss = settle_money(m);
    if (ss != MM_OK) return ss;
    if (!enable) {
        MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
        cudaFree(m->shadow32);
        m->shadow32 = nullptr;
        return MM_OK;
    }
    if (!m->shadow32)
        MM_CUDA_TRY(cudaMalloc(&m->shadow32, sizeof(float) * (2 * (size_t)m->T * m->S + m->S)),
                    "allocate FP32 shadow accumulators");
    return m->has_schedule ? shadow_init(m) : MM_OK;
}

mm_status mm_get_fp32_shadow_npv(mm_model *m, double *npv_host) {
    if (!m || !npv_host) return set_error(MM_ERR_INVALID_ARG, "NULL argument");
    if (!m->shadow32) return set_error(MM_ERR_STATE, "FP32 shadow accumulators are off");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    mm_status ss = settle_money(m);
    if (ss != MM_OK) return ss;
    std::vector<float> v(m->S);
    MM_CUDA_TRY(cudaMemcpyAsync(v.data(), m->shadow32 + 2 * (size_t)m->T * m->S, sizeof(float) * m->S,
                                cudaMemcpyDeviceToHost, m->stream),
                "read FP32 shadow NPV");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    for (int s = 0; s < m->S; s++) npv_host[s] = (double)v[s];
    return read_sticky(m);
}

mm_status mm_last_apply(mm_model *m, int32_t *applied, double *mean, double *sd) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (m->has_schedule) {
        mm_status st = settle_money(m);
        if (st == MM_OK) st = npv_stats_launch(m);
        if (st != MM_OK) return st;
    }
    // the result and the sticky status come back with one synchronisation
    MM_CUDA_TRY(cudaMemcpyAsync(m->apply_res_host, m->apply_res, sizeof(ApplyResult), cudaMemcpyDeviceToHost, m->stream),
                "read apply result");
    MM_CUDA_TRY(cudaMemcpyAsync(m->status_host, m->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, m->stream),
                "read status");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    if (applied) *applied = m->apply_res_host->applied;
    if (mean) *mean = m->apply_res_host->mean;
    if (sd) *sd = m->apply_res_host->std;
    return sticky_status(m, *m->status_host);
}

mm_status mm_npv(mm_model *m, double *npv_host, double *mean, double *sd) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    mm_status ss = settle_money(m);
    if (ss != MM_OK) return ss;
    std::vector<double> v(m->S);
    MM_CUDA_TRY(cudaMemcpyAsync(v.data(), m->npv, sizeof(double) * m->S, cudaMemcpyDeviceToHost, m->stream), "read npv");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    if (npv_host) std::memcpy(npv_host, v.data(), sizeof(double) * m->S);
    double mu = 0.0;
    for (double x : v) mu += x;
    mu /= m->S;
    double var = 0.0;
    for (double x : v) var += (x - mu) * (x - mu);
    if (mean) *mean = mu;
    if (sd) *sd = std::sqrt(var / m->S);
    return read_sticky(m);
}

mm_status mm_get_ore(mm_model *m, uint32_t *ore_host) {
    if (!m || !ore_host) return set_error(MM_ERR_INVALID_ARG, "NULL argument");
    MM_CUDA_TRY(cudaMemcpy2DAsync(ore_host, sizeof(uint32_t) * m->W, m->val + m->ore_off, sizeof(float) * m->R,
                                  sizeof(uint32_t) * m->W, m->B, cudaMemcpyDeviceToHost, m->stream), "read ore");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    return MM_OK;
}

mm_status mm_get_values(mm_model *m, float *value_host) {
    if (!m || !value_host) return set_error(MM_ERR_INVALID_ARG, "NULL argument");
    MM_CUDA_TRY(cudaMemcpy2DAsync(value_host, sizeof(float) * m->S, m->val, sizeof(float) * m->R, sizeof(float) * m->S,
                                  m->B, cudaMemcpyDeviceToHost, m->stream), "read values");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    return MM_OK;
}

mm_status mm_get_tonnage(mm_model *m, int64_t *mined_host, int64_t *ore_t_host) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    if (mined_host)
        MM_CUDA_TRY(cudaMemcpyAsync(mined_host, m->minedT, sizeof(int64_t) * m->T, cudaMemcpyDeviceToHost, m->stream),
                    "read mined");
    if (ore_t_host)
        MM_CUDA_TRY(cudaMemcpyAsync(ore_t_host, m->oreT, sizeof(int64_t) * (size_t)m->T * m->S, cudaMemcpyDeviceToHost,
                                    m->stream), "read ore tonnage");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    return MM_OK;
}

mm_status mm_get_metal(mm_model *m, double *metal_host) {
    if (!m || !metal_host) return set_error(MM_ERR_INVALID_ARG, "NULL argument");
    if (!m->has_schedule) return set_error(MM_ERR_STATE, "no schedule installed");
    mm_status ss = settle_money(m);
    if (ss != MM_OK) return ss;
    MM_CUDA_TRY(cudaMemcpyAsync(metal_host, m->metal, sizeof(double) * (size_t)m->T * m->S, cudaMemcpyDeviceToHost,
                                m->stream), "read metal");
    MM_CUDA_TRY(cudaStreamSynchronize(m->stream), "synchronize");
    return MM_OK;
}

}  // extern "C"
