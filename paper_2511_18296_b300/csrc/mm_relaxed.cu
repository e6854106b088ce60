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
// Forward: the two skinny contractions over blocks run on the fifth-generation
// tensor cores (tcgen05 kind::tf32 with each FP32 operand split into hi + lo,
// FP32-accurate; accumulators and the grade-side operand in tensor memory) --
// one warp-specialised CTA per SM takes a range of blocks and a tile of
// periods -- and the range partials are added by compensated FP32 in range
// order (deterministic), then the penalty, NPV_s and J in FP64.  O[t][s] is kept as the checkpoint the adjoint reads, so the
// backward pass never redoes the contraction.  The smoothed penalty and its
// derivative evaluate the exponential and logarithm in FP32 on an argument
// formed in FP64.
// Adjoint: with w_s = dJ/dNPV_s and c[t][s] = w_s P_t'(O[t][s]),
//   dJ/dx[b][t] = d_t (sum_s w_s v[b][s] - m_b sum_s c[t][s] ore[b][s]),
//   dJ/dg[b][s] = w_s ore[b][s] m_b price recovery sum_t d_t x[b][t];
// the sum over scenarios against c is again a TF32 product on the tensor
// cores (m16n8k8 from registers; ore is exact in TF32).  FP64 runs at a small fraction of the FP32
// rate on this part, so only sums and differences that need it are FP64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mm_internal.cuh"
#include "mm_umma.cuh"

namespace mm {

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

constexpr int kFwdSW = 128;     // scenarios per CTA (at most)

// d += a b for one 16 x 8 x 8 TF32 tile with FP32 accumulation, warp-wide:
// a holds A[gid][tig], A[gid + 8][tig], A[gid][tig + 4], A[gid + 8][tig + 4],
// b holds B[tig][gid], B[tig + 4][gid], d holds D[gid][2 tig], D[gid][2 tig + 1],
// D[gid + 8][2 tig], D[gid + 8][2 tig + 1] (gid = lane / 4, tig = lane % 4).
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// TF32 pieces of an FP32 value without a conversion instruction: hi = x on
// the TF32 grid (ten explicit mantissa bits; half a TF32 unit added to the
// magnitude, so ties go away from zero), lo = x - hi, exact in FP32.  The MMA
// reads lo truncated to TF32, an error below 2^-21 |x| of either sign.
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
    hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void cp_async16z(void *dst, const void *src, bool full) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(full ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4z(void *dst, const void *src, bool full) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(full ? 4 : 0)
                 : "memory");
}

// n / d for the small n of the copy loops: for d >= 2, m = floor((2^32 - 1) / d)
// + 1 = (2^32 + e) / d with 0 <= e < d fits 32 bits, and the high word of n m
// is n / d + n e / (d 2^32), exact whenever n d < 2^32; m = 0 marks d = 1.
__host__ __device__ inline uint32_t fdiv_magic(uint32_t d) { return d > 1u ? 0xffffffffu / d + 1u : 0u; }
__device__ __forceinline__ uint32_t fdiv(uint32_t n, uint32_t magic) { return magic ? __umulhi(n, magic) : n; }

// Forward contraction on the fifth-generation tensor cores (tcgen05), warp
// specialised.  One CTA per SM owns a contiguous range of whole 32-block
// tiles and a scenario tile of up to 128 (the MMA's M; the accumulator rows
// past the tile are never written out) for one tile of N periods from t0.
// Its warps:
//   * four copy warps stage tile k into one of kUmStages stages by cp.async,
//     each thread arriving on the stage's "full" mbarrier when its copies
//     have landed: 16-byte chunks of one contiguous stretch when the scenario
//     tile is the whole row (likewise x when the period tile is all periods),
//     else 16-byte chunks per row, else (rows not 16-byte aligned) elements;
//     1-D bulk (TMA) copies measured at about 16 bytes per clock per SM here,
//     well short of an SM's share of DRAM bandwidth, so they are not used;
//   * sixteen A warps, thread (m, q) for scenario row m and quarter q of the
//     tile's blocks: v' (model rows: v) split into TF32 hi + lo and the 0/1 ore flag,
//     stored into one of two operand buffers in TENSOR memory (lane m, one
//     column per block), where the MMA reads its A operand: the only operand
//     the tensor core reads from shared memory is the small B;
//   * two B warps, lane n for period n and half h of the blocks: y = x m
//     (model rows: also x) split into hi + lo, written into shared memory in
//     the tensor core's K-major layout (8-row x 16-byte core matrices);
//   * an MMA warp: one lane issues the tile's products, three per K step of
//     eight blocks with yh and yl side by side as one B of 2 N rows
//     (vh [yh | yl], o [yh | yl], vl yh), into FP32 accumulators in tensor
//     memory, and commits them to the operand buffer's "empty" mbarrier.
//     Even and odd K steps go to two accumulator sets (six accumulators);
//     V = (vh yh + vh yl + vl yh) and O = (o yh + o yl) are summed from them
//     at the end.  A single-CTA microbenchmark measured about 60 clocks per
//     kind::tf32 MMA issued from one thread with one set or two: the issue,
//     not the accumulator dependences, paces the products.
// Stages and buffers pass between the roles through mbarriers only (a stage
// is refilled after both preparing roles read it, a buffer rewritten after
// its products completed), so copies, operand preparation and products of
// consecutive tiles overlap.  Blocks past the last block of the range enter
// the products as zeros.  At the end the A warps read the accumulators (one
// scenario row per lane) and write the CTA's partial; the partials are added
// in range order afterwards (deterministic).  Every wait is bounded: on
// expiry the sticky timeout bit is raised and the CTA stops; the copies in
// flight are waited for and the tensor memory is always released.
constexpr int kUmBT = 32;        // blocks per tile: four K steps of eight
constexpr int kUmStages = 8;     // staged tiles
constexpr int kUmBufs = 2;       // operand buffers
constexpr int kUmM = 128;        // MMA M: scenarios per CTA
// Tensor memory (all 512 columns; one CTA per SM): two accumulator sets
// (even and odd K steps), each [Vh: vh [yh | yl], 2 N][O: o [yh | yl], 2 N]
// [Vl: vl yh, N], then the A buffers [buffer][vh, vl, o][kUmBT columns].
constexpr uint32_t kUmNCols = 512;
constexpr uint32_t kUmACol = 320;
constexpr int kUmAWarps = 16, kUmBWarps = 2;  // A: quarters of a tile's blocks per row, B: halves
constexpr int kUmCopyWarps = 4;
constexpr int kUmCopyWarp = kUmAWarps + kUmBWarps, kUmMmaWarp = kUmCopyWarp + kUmCopyWarps;
constexpr int kUmThreads = 32 * (kUmMmaWarp + 1);  // 736
constexpr long long kUmWait = 4000000000LL;        // clock cycles (about 2 s)

// Copy modes of the forward's stages.
struct UmCopy {
    int32_t g_rows;   // grade / value rows in 16-byte chunks (16-byte aligned)
    int32_t g_whole;  // ... the tile's rows as one contiguous stretch (scenario tile = whole row)
    int32_t x_rows;   // x rows in 16-byte chunks
    int32_t x_whole;  // ... the tile's x rows as one contiguous stretch (period tile = all periods)
};

struct UmLayout {
    int rw, ow, xs;  // staged grade-row stride, ore-word column (model rows), staged x-row stride
    size_t stg_g, stg_x, stg_m, opB, floats;
};
// sw: scenarios of the tile, zs: scenario tiles, R: model row length (floats).
__host__ __device__ inline UmLayout um_layout(int sw, int zs, int N, int T, int R, bool rows) {
    UmLayout L;
    const int c4 = (sw + 3) / 4 * 4;
    if (rows) {
        L.rw = zs == 1 ? R : c4 + 4;
        L.ow = zs == 1 ? -1 : c4;  // whole rows: the ore words at the model's own offset
    } else {
        L.rw = c4;
        L.ow = c4;
    }
    L.xs = T <= N ? (T + 3) / 4 * 4 : N;
    size_t off = 0;
    L.stg_g = off; off += (size_t)kUmStages * kUmBT * L.rw;
    L.stg_x = off; off += (size_t)kUmStages * kUmBT * L.xs;
    L.stg_m = off; off += (size_t)kUmStages * kUmBT;
    off = (off + 31) / 32 * 32;                                       // 128-byte aligned operands
    L.opB = off; off += (size_t)kUmBufs * (rows ? 4 : 2) * N * kUmBT; // [buffer][yh, yl (, xh, xl)][N x kUmBT]
    L.floats = off;
    return L;
}

// Arrive once on an mbarrier when all of this thread's earlier cp.async
// copies have completed (the expected count includes this arrival).
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(umma_saddr(bar)) : "memory");
}
// 16-byte cp.async to a shared-memory address (both 16-byte aligned).
__device__ __forceinline__ void cp_async16_sa(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma_saddr(bar)) : "memory");
}
template <typename G, int N, bool THR>
__global__ void __launch_bounds__(kUmThreads, 1) k_relax_fwd_umma(const float *__restrict__ x, const G *__restrict__ g,
                                                                   RelaxRows Rw, const uint32_t *__restrict__ mass,
                                                                   int32_t B, int32_t S, int32_t T, int32_t t0,
                                                                   RelaxEcon E, UmCopy C, float *__restrict__ part_o,
                                                                   float *__restrict__ part_v, uint32_t *status,
                                                                   int32_t stall, long long wait) {
    constexpr bool ROWS = sizeof(G) == sizeof(double);
    constexpr int KC = kUmBT / 4;  // 16-byte chunks of an operand row
    constexpr int KH = KC / 2;     // chunks per half tile
    constexpr uint32_t IDESC1 = umma_idesc_tf32(kUmM, N), IDESC2 = umma_idesc_tf32(kUmM, 2 * N);
    constexpr uint32_t SETC = 5 * N;  // columns of one accumulator set
    static_assert(2 * SETC <= kUmACol && kUmACol + kUmBufs * 3 * kUmBT <= kUmNCols, "tensor-memory columns");
    constexpr int NPREP = 32 * (kUmAWarps + kUmBWarps);  // threads that read a stage and write operands
    static_assert(N == 16 || N == 32, "N: a multiple of 16 for M = 128");
    static_assert(kUmAWarps == 16 && kUmBWarps == 2 && kUmBT == 32, "A: four quarters, B: two halves of a tile");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    extern __shared__ __align__(1024) float sm_um[];
    __shared__ __align__(8) uint64_t s_full[kUmStages], s_empty[kUmStages], s_opfull[kUmBufs], s_opempty[kUmBufs];
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;
    const int r = blockIdx.x, nr = gridDim.x;
    const int tiles = (B + kUmBT - 1) / kUmBT;
    const int k_lo = (int)((int64_t)r * tiles / nr), k_hi = (int)((int64_t)(r + 1) * tiles / nr);
    const int b_lo = k_lo * kUmBT, b_hi = min(B, k_hi * kUmBT), ntiles = k_hi - k_lo;
    const int s0 = blockIdx.z * kFwdSW, sw = min(kFwdSW, S - s0);
    const UmLayout L = um_layout(sw, (int)gridDim.z, N, T, Rw.R, ROWS);
    const int ow = L.ow < 0 ? Rw.ore_off : L.ow;
    float *stg_g = sm_um + L.stg_g, *stg_x = sm_um + L.stg_x;
    uint32_t *stg_m = reinterpret_cast<uint32_t *>(sm_um + L.stg_m);
    float *opB = sm_um + L.opB;
    const int nt = min(N, T - t0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // ---- copies (warps kUmCopyWarp ..): tile k into stage k mod kUmStages,
    // 16-byte cp.async chunks spread over the copy warps' threads ----
    const bool is_copy = warp >= kUmCopyWarp && warp < kUmCopyWarp + kUmCopyWarps;
    constexpr int NCP = 32 * kUmCopyWarps;
    const int ct = tid - 32 * kUmCopyWarp;
    const int c4 = (sw + 3) / 4 * 4;
    const int gcpr = ROWS ? c4 / 4 + 1 : sw / 4;  // 16-byte chunks of a row (per-row copies)
    // magic divisors only for the per-row and element copies
    const uint32_t gmag = (!is_copy || C.g_whole) ? 0u : fdiv_magic(C.g_rows ? gcpr : sw);
    const uint32_t xmag = (!is_copy || C.x_whole) ? 0u : fdiv_magic(C.x_rows ? nt / 4 : nt);
    const float *gf = ROWS ? Rw.val : reinterpret_cast<const float *>(g);
    const int glen = ROWS ? Rw.R : S;  // floats per source row
    auto issue_tile = [&](int k) {
        const int st = k % kUmStages, bb0 = b_lo + k * kUmBT, nb = min(kUmBT, b_hi - bb0);
        float *sg = stg_g + (size_t)st * kUmBT * L.rw, *sx = stg_x + (size_t)st * kUmBT * L.xs;
        const float *gt = gf + (size_t)bb0 * glen;
        if (C.g_whole) {  // the tile's rows are one contiguous stretch
            const int n16 = nb * glen / 4;
            const uint32_t d0 = umma_saddr(sg);
            for (int i = ct; i < n16; i += NCP) cp_async16_sa(d0 + 16u * i, gt + 4 * i);
        } else if (C.g_rows) {
            for (int i = ct; i < nb * gcpr; i += NCP) {
                const int j = (int)fdiv((uint32_t)i, gmag), q = i - j * gcpr;
                const float *row = gt + (size_t)j * glen;
                if (ROWS && q == gcpr - 1) cp_async16z(sg + j * L.rw + ow, row + Rw.ore_off + s0 / 32, true);
                else cp_async16z(sg + j * L.rw + 4 * q, row + s0 + 4 * q, true);
            }
        } else {
            for (int i = ct; i < nb * sw; i += NCP) {
                const int j = (int)fdiv((uint32_t)i, gmag), q = i - j * sw;
                cp_async4z(sg + j * L.rw + q, gt + (size_t)j * glen + s0 + q, true);
            }
        }
        const float *xt = x + (size_t)bb0 * T;
        if (C.x_whole) {
            const int n16 = nb * T / 4;
            const uint32_t d0 = umma_saddr(sx);
            for (int i = ct; i < n16; i += NCP) cp_async16_sa(d0 + 16u * i, xt + 4 * i);
        } else if (C.x_rows) {
            const int xcpr = nt / 4;
            for (int i = ct; i < nb * xcpr; i += NCP) {
                const int j = (int)fdiv((uint32_t)i, xmag), q = i - j * xcpr;
                cp_async16z(sx + j * L.xs + 4 * q, xt + (size_t)j * T + t0 + 4 * q, true);
            }
        } else {
            for (int i = ct; i < nb * nt; i += NCP) {
                const int j = (int)fdiv((uint32_t)i, xmag), q = i - j * nt;
                cp_async4z(sx + j * L.xs + q, xt + (size_t)j * T + t0 + q, true);
            }
        }
        if (ct < kUmBT) cp_async4z(&stg_m[st * kUmBT + ct], mass + bb0 + (ct < nb ? ct : 0), ct < nb);
    };
    // tile 0's copies go out before the set-up below (they need no barrier;
    // the stage's arrival comes after it), so their latency overlaps it
    if (is_copy && ntiles > 0) issue_tile(0);
    if (tid == 0) {
        for (int i = 0; i < kUmStages; i++) {
            // one cp.async arrival per copy thread (test-only stall: one more, which never comes)
            umma_bar_init(&s_full[i], 32 * kUmCopyWarps + (stall ? 1 : 0));
            umma_bar_init(&s_empty[i], NPREP);
        }
        for (int i = 0; i < kUmBufs; i++) {
            umma_bar_init(&s_opfull[i], NPREP);
            umma_bar_init(&s_opempty[i], 1);
        }
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) umma_alloc(&s_tmem, kUmNCols);
    umma_fence_before();
    __syncthreads();
    umma_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *err = &s_err;
    if (is_copy) {
        for (int k = 0; k < ntiles; k++) {
            const int st = k % kUmStages;
            if (k >= kUmStages && !umma_bar_wait(&s_empty[st], (uint32_t)(k / kUmStages - 1) & 1u, wait)) *err = 1;
            if (*err) break;
            if (k > 0) issue_tile(k);
            cp_async_arrive(&s_full[st]);  // when this thread's copies so far (tile k's and earlier) have landed
        }
        asm volatile("cp.async.wait_all;" ::: "memory");  // nothing lands in shared memory after the CTA ends
    } else if (warp < kUmAWarps + kUmBWarps) {
        // ---- operands: A warps (thread (m, h) = scenario row m, quarter h of
        // the blocks), B warps (lane n = period n, half h of the blocks) ----
        const bool isA = warp < kUmAWarps;
        const int row_id = isA ? (tid & (kUmM - 1)) : lane;
        const int h = isA ? warp / 4 : warp - kUmAWarps;  // A: quarter, B: half
        const int base = (((row_id >> 3) * KC) * 8 + (row_id & 7)) * 4;  // B: chunk c at base + 32 c
        const float c1 = E.pf * E.rf, pcm = E.pcf + E.mcf, mcn = -E.mcf;
        const uint32_t one = __float_as_uint(1.0f);
        // A: this warp's lanes (32 (warp mod 4) ..) and quarter of the columns
        const uint32_t ta0 = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + kUmACol + 8u * (isA ? h : 0);
        for (int k = 0; k < ntiles; k++) {
            const int st = k % kUmStages, bsel = k % kUmBufs, nb = min(kUmBT, b_hi - (b_lo + k * kUmBT));
            bool ok = umma_bar_wait(&s_full[st], (uint32_t)(k / kUmStages) & 1u, wait);
            if (ok && k >= kUmBufs) ok = umma_bar_wait(&s_opempty[bsel], (uint32_t)(k / kUmBufs - 1) & 1u, wait);
            if (!ok) *err = 1;
            if (__any_sync(0xffffffffu, *err != 0)) break;  // warp-uniform: tcgen05.st is warp-collective
            umma_fence_after();
            if (isA) {
                // A row m only enters D row m, and D rows past the scenario
                // tile are never read: those rows take whatever the stage holds.
                // Blocks past the range (the ragged last tile) enter as zeros.
                const float *sg = stg_g + (size_t)st * kUmBT * L.rw + (size_t)(8 * h) * L.rw + row_id;
                float gvs[8];
                uint32_t ows[ROWS ? 8 : 1];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    gvs[i] = sg[i * L.rw];
                    if (ROWS) ows[i] = __float_as_uint(sg[i * L.rw + ow - row_id + (row_id >> 5)]);
                }
                uint32_t hi[8], lo[8], o[8];
                const int nlive = nb - 8 * h;  // >= 8 except in the ragged last tile
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const float gv = gvs[i];
                    bool ore;
                    float val;
                    if (ROWS) {
                        ore = (ows[ROWS ? i : 0] >> (row_id & 31)) & 1u;
                        val = gv;
                    } else {
                        ore = THR ? gv >= E.g_thr : relax_ore(gv, E);
                        val = ore ? fmaf(gv, c1, -pcm) : mcn;
                    }
                    if (nlive < 8 && i >= nlive) {
                        ore = false;
                        val = 0.0f;
                    }
                    tf32_split(val, hi[i], lo[i]);
                    o[i] = ore ? one : 0u;
                }
                const uint32_t ta = ta0 + (uint32_t)(bsel * 3 * kUmBT);
                umma_st8(ta, hi);
                umma_st8(ta + kUmBT, lo);
                umma_st8(ta + 2 * kUmBT, o);
                umma_wait_st();
            } else if (row_id < N) {
                const float *sx = stg_x + (size_t)st * kUmBT * L.xs + row_id;
                const uint32_t *smm = stg_m + st * kUmBT;
                float *B0 = opB + (size_t)bsel * (ROWS ? 4 : 2) * N * kUmBT + base, *B1 = B0 + N * kUmBT;
                float *B2 = B1 + N * kUmBT, *B3 = B2 + N * kUmBT;
                float xvs[4 * KH], mvs[4 * KH];
#pragma unroll
                for (int i = 0; i < 4 * KH; i++) {
                    const int j = 4 * KH * h + i;
                    xvs[i] = j < nb ? sx[j * L.xs] : 0.0f;  // B row n only enters D column n (n >= nt unread)
                    mvs[i] = (float)smm[j];
                }
#pragma unroll
                for (int cc = 0; cc < KH; cc++) {
                    const int c = h * KH + cc;
                    uint32_t yh[4], yl[4], xh[4], xl[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const float xv = xvs[4 * cc + e];
                        tf32_split(xv * mvs[4 * cc + e], yh[e], yl[e]);
                        if (ROWS) tf32_split(xv, xh[e], xl[e]);
                    }
                    *reinterpret_cast<uint4 *>(B0 + 32 * c) = make_uint4(yh[0], yh[1], yh[2], yh[3]);
                    *reinterpret_cast<uint4 *>(B1 + 32 * c) = make_uint4(yl[0], yl[1], yl[2], yl[3]);
                    if (ROWS) {
                        *reinterpret_cast<uint4 *>(B2 + 32 * c) = make_uint4(xh[0], xh[1], xh[2], xh[3]);
                        *reinterpret_cast<uint4 *>(B3 + 32 * c) = make_uint4(xl[0], xl[1], xl[2], xl[3]);
                    }
                }
            }
            if (isA) umma_fence_before();  // tensor-memory stores -> the MMA thread
            else umma_fence_operands();    // shared-memory stores -> the tensor core
            mbar_arrive(&s_empty[st]);
            mbar_arrive(&s_opfull[bsel]);
        }
    } else if (warp == kUmMmaWarp && lane == 0) {
        // ---- products: one lane issues every MMA of the CTA ----
        for (int k = 0; k < ntiles; k++) {
            const int bsel = k % kUmBufs, nb = min(kUmBT, b_hi - (b_lo + k * kUmBT));
            if (!umma_bar_wait(&s_opfull[bsel], (uint32_t)(k / kUmBufs) & 1u, wait)) *err = 1;
            if (*err) break;
            umma_fence_after();
            const float *B0 = opB + (size_t)bsel * (ROWS ? 4 : 2) * N * kUmBT;
            const uint32_t a0 = tmem + kUmACol + (uint32_t)(bsel * 3 * kUmBT), a1 = a0 + kUmBT, a2 = a1 + kUmBT;
            const uint32_t b0 = umma_saddr(B0), b2 = b0 + 8u * N * kUmBT;
#pragma unroll
            for (int s = 0; s < kUmBT / 8; s++) {
                if (8 * s >= nb) break;  // K steps past the range's last block add nothing
                // the first product into each set overwrites it
                const uint32_t acc = (k > 0 || s > 1) ? 1u : 0u, so = 256u * s, ka = 8u * s;
                const uint32_t dVh = tmem + (uint32_t)(s & 1) * SETC, dO = dVh + 2 * N, dVl = dVh + 4 * N;
                const uint64_t dBy = umma_sdesc(b0 + so, 128, KC * 128);               // [yh | yl], 2 N rows
                const uint64_t dBx = ROWS ? umma_sdesc(b2 + so, 128, KC * 128) : dBy;  // [xh | xl]
                const uint64_t dBxh = umma_sdesc((ROWS ? b2 : b0) + so, 128, KC * 128);  // xh (yh), N rows
                umma_tf32_ta(dVh, a0 + ka, dBx, IDESC2, acc);
                umma_tf32_ta(dO, a2 + ka, dBy, IDESC2, acc);
                umma_tf32_ta(dVl, a1 + ka, dBxh, IDESC1, acc);
            }
            umma_commit(&s_opempty[bsel]);
        }
    }
    // ---- the CTA's partial: warp w reads tensor-memory lanes 32 (w mod 4),
    // columns 16 (w / 4) .. + 15 of the accumulators ----
    if (warp < kUmAWarps) {
        bool ok = *err == 0;
        if (ntiles > 0 && ok &&
            !umma_bar_wait(&s_opempty[(ntiles - 1) % kUmBufs], (uint32_t)((ntiles - 1) / kUmBufs) & 1u, wait))
            ok = false;
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
        if (!ok && lane == 0) atomicOr(status, kStTimeout);
        umma_fence_after();
        const int m = 32 * (warp & 3) + lane, hc = warp >> 2;
        // the odd set holds products unless the range is one tile of at most 8 blocks
        const int nsets = (ntiles > 1 || b_hi - b_lo > 8) ? 2 : 1;
        if (16 * hc < N) {
            const bool have = ntiles > 0 && ok;
            float v[16], o[16];
            if (have) {
                const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 16u * hc;
                float a[16], b[16], c[16];
                for (int q = 0; q < 16; q++) v[q] = o[q] = 0.0f;
                for (int set = 0; set < nsets; set++) {
                    const uint32_t sb = base + (uint32_t)set * SETC;
                    umma_ld16(sb, a);          // vh yh
                    umma_ld16(sb + N, b);      // vh yl
                    umma_ld16(sb + 4 * N, c);  // vl yh
#pragma unroll
                    for (int q = 0; q < 16; q++) v[q] += (a[q] + b[q]) + c[q];
                    umma_ld16(sb + 2 * N, a);  // o yh
                    umma_ld16(sb + 3 * N, b);  // o yl
#pragma unroll
                    for (int q = 0; q < 16; q++) o[q] += a[q] + b[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const int t = 16 * hc + q;
                if (m < sw && t < nt) {
                    const size_t at = ((size_t)r * T + t0 + t) * S + s0 + m;
                    part_v[at] = have ? v[q] : 0.0f;
                    part_o[at] = have ? o[q] : 0.0f;
                }
            }
        }
    }
    umma_fence_before();
    __syncthreads();
    if (warp == 0) umma_dealloc(tmem, kUmNCols);
}

// CTAs per scenario tile of the forward: one per SM (each owns a range of
// blocks and writes one partial), at least one 32-block tile each.
static int relax_fwd_ctas(const mm_model *m, int B, int S) {
    const int zs = (S + kFwdSW - 1) / kFwdSW;
    return std::max(1, std::min((B + kUmBT - 1) / kUmBT, std::max(1, m->num_sms / zs)));
}

template <typename G>
static mm_status relax_fwd_launch(const mm_model *m, const float *x, const G *g, RelaxRows Rw, const uint32_t *mass,
                                  int32_t B, int32_t S, int32_t T, RelaxEcon E, float *part_o, float *part_v, int nr,
                                  cudaStream_t st, int stall) {
    const long long wait = stall ? 2000000LL : kUmWait;  // test-only stall: about 1 ms
    const int zs = (S + kFwdSW - 1) / kFwdSW;
    constexpr bool rows = sizeof(G) == sizeof(double);
    UmCopy C;
    if (rows) {
        if (((uintptr_t)Rw.val & 15u) != 0 || Rw.R % 4 != 0 || Rw.ore_off % 4 != 0) return MM_ERR_INVALID_ARG;
        C.g_rows = 1;
    } else {
        C.g_rows = (S % 4 == 0 && ((uintptr_t)g & 15u) == 0) ? 1 : 0;
    }
    C.g_whole = C.g_rows && zs == 1;
    C.x_rows = (T % 4 == 0 && ((uintptr_t)x & 15u) == 0) ? 1 : 0;  // period tiles start at multiples of 32
    for (int tb = 0; tb < T; tb += 32) {
        const int N = T - tb <= 16 ? 16 : 32;
        C.x_whole = C.x_rows && T <= N;
        // at least half of an SM's shared memory: one CTA per SM, which owns all of its tensor memory
        const size_t smem = std::max<size_t>(um_layout(std::min(S, kFwdSW), zs, N, T, Rw.R, rows).floats * sizeof(float),
                                             116u << 10);
        using Fn = void (*)(const float *, const G *, RelaxRows, const uint32_t *, int32_t, int32_t, int32_t, int32_t,
                            RelaxEcon, UmCopy, float *, float *, uint32_t *, int32_t, long long);
        Fn fn;
        if (E.use_thr) fn = N == 16 ? k_relax_fwd_umma<G, 16, true> : k_relax_fwd_umma<G, 32, true>;
        else fn = N == 16 ? k_relax_fwd_umma<G, 16, false> : k_relax_fwd_umma<G, 32, false>;
        MM_CUDA_TRY(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "forward smem");
        fn<<<dim3((unsigned)nr, 1, (unsigned)zs), kUmThreads, smem, st>>>(x, g, Rw, mass, B, S, T, tb, E, C, part_o,
                                                                          part_v, m->status, stall, wait);
        mm_status r = check_launch("k_relax_fwd_umma");
        if (r != MM_OK) return r;
    }
    return MM_OK;
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

// End of the forward pass, one launch over (32-scenario chunk, period):
//   1. O[t][s] and V[t][s] for the CTA's 32 scenarios of period t from the
//      range partials: warp w adds ranges w, w + kFinWarps, ... by compensated
//      FP32 sums (each load reads 32 consecutive floats of one partial; all of
//      a lane's loads are in flight together), and warps 0 (O) and 1 (V)
//      merge the warp sums in warp order (deterministic; the error is about
//      one FP32 rounding of the total, no FP64 on the long sums);
//   2. the FP64 checkpoint O[t][s] and term[t][s] = d_t (V - P_t(O)), with
//      (Q_t - O) / m_ref formed in FP64 and the two softplus branches in FP32;
//   3. the last CTA (release-acquire ticket) forms every NPV_s = sum_t
//      term[t][s] by fixed pairwise trees over the periods, the (sum, sum of
//      squares) over scenarios by fixed trees, the mean, the population std
//      and J, and resets the ticket.
// For the adjoint it also leaves P_t'(O[t][s]) (step 2) and the scenario
// weights per unit upstream gradient, 1/S - lambda (NPV_s - mean) / (S std)
// (step 3), both FP32, so a backward pass on these outputs needs no
// coefficient launch.
// A warp-wide FP64 instruction issues about every 16 clocks per SM on this
// part, so step 3 spends FP64 only where there are scenarios: the trees skip
// the additions of the zero padding past T (exact, so the sums are those of
// the full trees) and warps without scenarios skip the reductions.  A split
// of step 3 over one CTA per chunk and a second ticket measured slower: the
// extra fence, ticket and load round trips cost more than the FP64 saved.
constexpr int kFinWarps = 16;
constexpr int kFinBatch = 10;  // partial loads in flight per lane and array

__device__ __forceinline__ float relax_softplus_f(float bz) { return fmaxf(bz, 0.0f) + log1pf(expf(-fabsf(bz))); }

// sum of q[0 .. 31] by a fixed pairwise tree, q[i] = 0 for i >= n: pairs of
// two padding zeros are not added (x + 0 = x, so the result is the full tree's)
__device__ __forceinline__ double relax_tree32(const double (&q)[32], int n) {
    double a[16];
#pragma unroll
    for (int u = 0; u < 16; u++) a[u] = 2 * u + 1 < n ? q[2 * u] + q[2 * u + 1] : q[2 * u];
#pragma unroll
    for (int w = 8, span = 2; w > 0; w >>= 1, span <<= 1)  // a[v] covers q[span v .. span v + span - 1]
#pragma unroll
        for (int u = 0; u < w; u++) a[u] = (2 * u + 1) * span < n ? a[2 * u] + a[2 * u + 1] : a[2 * u];
    return a[0];
}

__global__ void __launch_bounds__(32 * kFinWarps, 1) k_relax_finish(const float *__restrict__ part_o,
                                                                const float *__restrict__ part_v, int32_t nr,
                                                                int32_t S, int32_t T, const double *__restrict__ disc,
                                                                const uint64_t *__restrict__ target, RelaxEcon E,
                                                                double *__restrict__ o_out, double *term,
                                                                uint32_t *tick, double *__restrict__ npv,
                                                                double *__restrict__ J, float *__restrict__ dp_out,
                                                                float *__restrict__ wt_out) {
    __shared__ float s_sum[2][kFinWarps][32], s_cmp[2][kFinWarps][32];  // [O / V][warp][lane]
    __shared__ float s_vm[2][32];                                         // V merged by warp 1: (sum, compensation)
    __shared__ double s_red[2][kFinWarps];
    __shared__ double s_mv[2];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chunk = blockIdx.x, t = blockIdx.y;
    const int s = 32 * chunk + lane;
    const size_t TS = (size_t)T * S, col = (size_t)t * S + s;
    // a backward launched next (as this grid's programmatic dependent) may
    // start staging its grades now; it waits for this grid before it reads
    // anything this grid writes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // the period's inputs are not written by the forward: read before the wait
    const double Qt = (double)target[t], dt = disc[t];
    // launched as a programmatic dependent of the forward contraction: wait
    // until its grid has completed and its partials are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    float so = 0.0f, co = 0.0f, sv = 0.0f, cv = 0.0f;
    if (s < S) {
        for (int c0 = warp; c0 < nr; c0 += kFinBatch * kFinWarps) {
            float a[kFinBatch], b[kFinBatch];
#pragma unroll
            for (int u = 0; u < kFinBatch; u++) {
                const int c = c0 + kFinWarps * u;
                a[u] = c < nr ? __ldcg(part_o + (size_t)c * TS + col) : 0.0f;
                b[u] = c < nr ? __ldcg(part_v + (size_t)c * TS + col) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < kFinBatch; u++)
                if (c0 + kFinWarps * u < nr) {  // warp-uniform: only the ranges that exist
                    relax_neumaier(so, co, a[u]);
                    relax_neumaier(sv, cv, b[u]);
                }
        }
    }
    s_sum[0][warp][lane] = so;
    s_cmp[0][warp][lane] = co;
    s_sum[1][warp][lane] = sv;
    s_cmp[1][warp][lane] = cv;
    __syncthreads();
    if (warp < 2) {  // warp 0 merges O, warp 1 merges V, each in warp order
        float sm = s_sum[warp][0][lane], cm = s_cmp[warp][0][lane];
        for (int w = 1; w < kFinWarps; w++) relax_merge(sm, cm, s_sum[warp][w][lane], s_cmp[warp][w][lane]);
        if (warp == 1) {
            s_vm[0][lane] = sm;
            s_vm[1][lane] = cm;
        } else {
            so = sm;
            co = cm;
        }
    }
    __syncthreads();
    if (warp == 0) {
        if (s < S) {
            sv = s_vm[0][lane];
            cv = s_vm[1][lane];
            const double O = (double)so + (double)co, V = (double)sv + (double)cv;
            o_out[col] = O;
            const float bz = (float)E.beta * (float)((Qt - O) * E.inv_mref);
            const float pen = (float)(E.a * E.m_ref * E.inv_beta) * relax_softplus_f(bz) +
                              (float)(E.e * E.m_ref * E.inv_beta) * relax_softplus_f(-bz);
            term[col] = dt * (V - (double)pen);
            // P_t'(O) for the adjoint: -a sigma(beta (Q - O) / m_ref) + e sigma(beta (O - Q) / m_ref)
            dp_out[col] = -(float)E.a / (1.0f + expf(-bz)) + (float)E.e / (1.0f + expf(bz));
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(tick, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last CTA: NPV_s for every scenario (32 periods at a time, all loads
    // in flight, each batch by a fixed pairwise tree, the batch sums in period
    // order), then (sum, sum of squares) by fixed trees over lanes and warps;
    // warps past the last scenario hold zeros and skip the FP64 work
    const int nw = min(kFinWarps, (S + 31) / 32);  // warps holding scenarios (of the first pass)
    double x1 = 0.0, x2 = 0.0;
    double mine0 = 0.0, mine1 = 0.0;  // this thread's first two NPV_s, kept for the weights below
    for (int sc = threadIdx.x, r = 0; sc < S; sc += blockDim.x, r++) {
        double acc = 0.0;
        for (int t0 = 0; t0 < T; t0 += 32) {
            double q[32];
#pragma unroll
            for (int u = 0; u < 32; u++) q[u] = t0 + u < T ? __ldcg(term + (size_t)(t0 + u) * S + sc) : 0.0;
            acc += relax_tree32(q, T - t0);
        }
        npv[sc] = acc;
        if (r == 0) mine0 = acc;
        else if (r == 1) mine1 = acc;
        x1 += acc;
        x2 += acc * acc;
    }
    if (warp < nw) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            x1 += __shfl_xor_sync(0xffffffffu, x1, off);
            x2 += __shfl_xor_sync(0xffffffffu, x2, off);
        }
    }
    if (lane == 0) {
        s_red[0][warp] = x1;
        s_red[1][warp] = x2;
    }
    __syncthreads();
    if (warp == 0) {
        double y1 = lane < nw ? s_red[0][lane] : 0.0, y2 = lane < nw ? s_red[1][lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            if (off < nw) {  // lanes >= nw hold zeros: the levels above add only zeros
                y1 += __shfl_xor_sync(0xffffffffu, y1, off);
                y2 += __shfl_xor_sync(0xffffffffu, y2, off);
            }
        }
        if (lane == 0) {
            const double mean = y1 * E.inv_S;
            const double var = fmax(y2 * E.inv_S - mean * mean, 0.0);
            // the std to FP32 accuracy (a relative 1e-7 of lambda std in J)
            J[0] = mean - E.lambda * (double)sqrtf((float)var);
            s_mv[0] = mean;
            s_mv[1] = var > 0.0 ? E.lambda * E.inv_S * (double)rsqrtf((float)var) : 0.0;
            *tick = 0u;  // every CTA has taken its ticket
        }
    }
    __syncthreads();
    // the adjoint's scenario weights per unit gJ: 1/S - lambda (NPV_s - mean) / (S std)
    for (int sc = threadIdx.x, r = 0; sc < S; sc += blockDim.x, r++)
        wt_out[sc] = (float)(E.inv_S - s_mv[1] * ((r == 0 ? mine0 : (r == 1 ? mine1 : __ldcg(npv + sc))) - s_mv[0]));
}

// Adjoint coefficients: w_s = gJ (1/S - lambda (NPV_s - mean) / (S std))
// (the std term dropped where std = 0) and c[t][s] = w_s P_t'(O[t][s]), one
// thread per (t, s) over many CTAs; every CTA forms mean and std itself, in
// one pass over NPV_s - NPV_0 (sum and sum of squares side by side), with the
// thread's own inputs loaded before that pass, and 1 / std in FP32.  Only what needs it is FP64
// (the scenario statistics, w_s and Q_t - O[t][s]); the sigmoids, a and e and
// the product are FP32 (c is stored in FP32).  The adjoint that reads c and w
// launches as this grid's programmatic dependent.
__global__ void __launch_bounds__(128) k_relax_coef(const double *__restrict__ npv, const double *__restrict__ o,
                                                    const uint64_t *__restrict__ target, const double *__restrict__ gJ,
                                                    int32_t S, int32_t T, int32_t Sp, RelaxEcon E,
                                                    float *__restrict__ w_out, float *__restrict__ c_out) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ double red[2][4];
    __shared__ double s_k[3];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = i < T * S;
    const int t = on ? i / S : 0, s = on ? i - t * S : 0;
    const double O = on ? o[i] : 0.0, Q = on ? (double)target[t] : 0.0, ns = npv[s], x0 = npv[0];
    double a1 = 0.0, a2 = 0.0;
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
        const double d = npv[k] - x0;
        a1 += d;
        a2 += d * d;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = a1;
        red[1][warp] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // one division per CTA: w_s = k0 - k1 ((NPV_s - NPV_0) - dm)
        const double A1 = (red[0][0] + red[0][1]) + (red[0][2] + red[0][3]);
        const double A2 = (red[1][0] + red[1][1]) + (red[1][2] + red[1][3]);
        // 1 / std to FP32 accuracy (w is stored in FP32)
        const double dm = A1 * E.inv_S, var = fmax(A2 * E.inv_S - dm * dm, 0.0), g = gJ[0];
        s_k[0] = g * E.inv_S;
        s_k[1] = var > 0.0 ? g * E.lambda * E.inv_S * (double)rsqrtf((float)var) : 0.0;
        s_k[2] = dm;
    }
    __syncthreads();
    if (!on) return;
    const double w = s_k[0] - s_k[1] * ((ns - x0) - s_k[2]);
    if (t == 0) w_out[s] = (float)w;
    const float bz = (float)E.beta * (float)((Q - O) * E.inv_mref);
    const float dp = -(float)E.a / (1.0f + expf(-bz)) + (float)E.e / (1.0f + expf(bz));
    c_out[(size_t)t * Sp + s] = (float)w * dp;
}

// Tiled adjoint on the tensor cores (the fast path).  With the period tile
// t0 .. t0 + TT - 1 (TT a multiple of 8, at most 32),
//   A[b][t] = sum_s ore[b][s] c[t][s]
// is an m16n8k8 TF32 product: ore is 0 or 1 (exact in TF32) and c is split
// into TF32 hi + lo (two products, FP32-accurate), so the tensor pipe does the
// B x S x TT contraction and the CUDA cores only turn grades into ore flags.
// Alongside, each lane sums its share of u_b = sum_s w_s v[b][s] (caller
// grades: v = m_b v', v' = ore ? g c1 - (pc + mc) : -mc) in FP32, and
//   dJ/dx[b][t] = d_t (u_b - m_b A[b][t]),
//   dJ/dg[b][s] = w_s ore[b][s] m_b price recovery sum_t d_t x[b][t]  (t0 == 0).
// CTA r owns a contiguous range of the blocks, in tiles of kAdjBT whose grade
// rows (or value rows and ore words), x rows and masses are copied into
// shared memory by cp.async one tile ahead (rows past the range zero-filled),
// so each grade is read from memory once; two warps share each 16-block M
// tile, one taking the even and one the odd K steps (eight scenarios each),
// and the odd one's sums are added to the even one's in that order through
// shared memory.  dJ/dg is written as one contiguous stretch per tile, four
// scenarios per lane, with streaming stores.  The coefficients come from
// k_relax_coef: this grid issues its first copies and only then waits for
// that launch (griddepcontrol.wait).
constexpr int kAdjBT = 64;       // blocks per staged tile
constexpr int kAdjKSplit = 2;  // warps sharing a 16-block M tile (halves of the K steps)
constexpr int kAdjWarps = kAdjBT / 16 * kAdjKSplit;
constexpr int kAdjStages = 2;
constexpr int kAdjMaxTT = 32;

struct AdjLayout {
    int K8, RS, XS;  // scenarios padded to 8; staged row stride (4 mod 8: conflict-free fragment
                     // loads); staged x row stride (0: not staged)
    size_t g, x, m, c, w, d, D, x2, floats;
};
__host__ __device__ inline AdjLayout adj_layout(int S, int T, int TT, bool rows, bool stage_x) {
    AdjLayout L;
    L.K8 = (S + 7) / 8 * 8;
    const int words = rows ? ((S + 31) / 32 + 3) / 4 * 4 : 0;  // ore words at column K8
    int rs = L.K8 + words;
    rs += (12 - rs % 8) % 8;
    L.RS = rs;
    L.XS = stage_x ? (T + 3) / 4 * 4 : 0;
    size_t off = 0;
    L.g = off; off += (size_t)kAdjStages * kAdjBT * L.RS;
    L.x = off; off += (size_t)kAdjStages * kAdjBT * L.XS;
    L.m = off; off += (size_t)kAdjStages * kAdjBT;
    L.c = off; off += (size_t)2 * L.K8 * TT;  // (hi, lo) of c in fragment order
    L.w = off; off += L.K8;
    L.d = off; off += (size_t)(T + 3) / 4 * 4;
    L.D = off; off += kAdjBT;
    L.x2 = off; off += (size_t)(kAdjBT / 16) * 32 * (TT / 2 + 2);  // the K halves' exchange
    L.floats = off;
    return L;
}

template <typename G, int TT, bool THR>
__global__ void __launch_bounds__(32 * kAdjWarps, 2) k_relax_adj_tc(const float *__restrict__ x, const G *__restrict__ g,
                                                               RelaxRows Rw, const uint32_t *__restrict__ mass,
                                                               const float *__restrict__ w, const float *__restrict__ c,
                                                               int32_t Sp, const double *__restrict__ gJs,
                                                               const double *__restrict__ disc, int32_t B,
                                                               int32_t S, int32_t T, int32_t t0, RelaxEcon E,
                                                               int32_t vec, int32_t xvec, int32_t gvec,
                                                               float *__restrict__ gx, float *__restrict__ gg) {
    constexpr bool ROWS = sizeof(G) == sizeof(double);
    static_assert(TT % 8 == 0 && TT <= kAdjMaxTT, "period tile");
    extern __shared__ __align__(16) float sm[];
    const bool want_g = gg != nullptr && t0 == 0;
    const bool xst = want_g && T <= kAdjMaxTT;  // x rows staged with the tile, else read from memory
    const AdjLayout L = adj_layout(S, T, TT, ROWS, xst);
    float *s_g = sm + L.g, *s_x = sm + L.x, *s_w = sm + L.w, *s_d = sm + L.d, *s_D = sm + L.D, *s_x2 = sm + L.x2;
    uint32_t *s_m = reinterpret_cast<uint32_t *>(sm + L.m);
    uint4 *s_c = reinterpret_cast<uint4 *>(sm + L.c);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nth = blockDim.x;
    const int gid = lane >> 2, tig = lane & 3;
    const int r = blockIdx.x, nr = gridDim.x;
    const int b_lo = (int)((int64_t)r * B / nr), b_hi = (int)((int64_t)(r + 1) * B / nr);
    const int ntiles = (b_hi - b_lo + kAdjBT - 1) / kAdjBT;
    const int nt = min(TT, T - t0);
    // scenario columns S .. K8 - 1 of the staged rows are never copied (only
    // K-padding of the products): zero them once
    if (L.K8 > S)
        for (int i = tid; i < kAdjStages * kAdjBT * (L.K8 - S); i += nth) {
            const int row = i / (L.K8 - S);
            s_g[(size_t)row * L.RS + S + (i - row * (L.K8 - S))] = 0.0f;
        }
    // copy chunks per staged row: grade / value chunks of four scenarios (or
    // single scenarios) and ore-word chunks; x chunks of four periods (or one)
    const int nv4 = (S + 3) / 4;
    const int gcs = ROWS ? nv4 + ((S + 31) / 32 + 3) / 4 : (vec ? S / 4 : S);
    const int xcs = xvec ? T / 4 : T;
    const uint32_t gmag = fdiv_magic(gcs), xmag = fdiv_magic(xcs);
    const uint32_t cmag = fdiv_magic(S / 4 > 0 ? S / 4 : 1), smag = fdiv_magic(S);
    auto issue = [&](int k) {
        const int st = k % kAdjStages, bb0 = b_lo + k * kAdjBT, nb = min(kAdjBT, b_hi - bb0);
        float *sg = s_g + (size_t)st * kAdjBT * L.RS;
        for (int i = tid; i < kAdjBT * gcs; i += nth) {
            const int j = (int)fdiv((uint32_t)i, gmag), q = i - j * gcs;
            const bool live = j < nb;
            const size_t b = (size_t)(bb0 + (live ? j : 0));
            float *dst = sg + j * L.RS;
            if (ROWS) {
                const float *row = Rw.val + b * Rw.R;
                if (q < nv4) cp_async16z(dst + 4 * q, row + 4 * q, live);
                else cp_async16z(dst + L.K8 + 4 * (q - nv4), row + Rw.ore_off + 4 * (q - nv4), live);
            } else if (vec) {
                cp_async16z(dst + 4 * q, reinterpret_cast<const float *>(g) + b * S + 4 * q, live);
            } else {
                cp_async4z(dst + q, reinterpret_cast<const float *>(g) + b * S + q, live);
            }
        }
        if (xst)
            for (int i = tid; i < kAdjBT * xcs; i += nth) {
                const int j = (int)fdiv((uint32_t)i, xmag), q = i - j * xcs;
                const bool live = j < nb;
                const float *xr = x + (size_t)(bb0 + (live ? j : 0)) * T;
                float *xd = s_x + ((size_t)st * kAdjBT + j) * L.XS;
                if (xvec) cp_async16z(xd + 4 * q, xr + 4 * q, live);
                else cp_async4z(xd + q, xr + q, live);
            }
        for (int j = tid; j < kAdjBT; j += nth)
            cp_async4z(&s_m[st * kAdjBT + j], mass + bb0 + (j < nb ? j : 0), j < nb);
    };
    for (int k = 0; k < kAdjStages - 1; k++) {
        if (k < ntiles) issue(k);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // the coefficients are the preceding launch's results: w_s and c[t][s]
    // from k_relax_coef, or (gJs set) the forward's weights per unit gJ and
    // P_t'(O[t][s]), scaled here: w_s = gJ wt_s, c[t][s] = w_s P_t'
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const float gsc = gJs ? (float)gJs[0] : 1.0f;
    for (int i = tid; i < L.K8; i += nth) s_w[i] = i < S ? gsc * w[i] : 0.0f;
    for (int i = tid; i < T; i += nth) s_d[i] = (float)disc[i];
    // c[t0 + n][s] split into TF32 pieces in fragment order: 16-byte word
    // ((q TT + n) 4 + i) holds hi and lo of scenarios 8q + i and 8q + i + 4
    for (int u = tid; u < (L.K8 / 8) * TT * 4; u += nth) {
        const int i = u & 3, qn = u >> 2, q = qn / TT, n = qn - q * TT;
        const int sa = 8 * q + i, sb = sa + 4;
        const bool on = n < nt;
        float ca = on && sa < S ? c[(size_t)(t0 + n) * Sp + sa] : 0.0f;
        float cb = on && sb < S ? c[(size_t)(t0 + n) * Sp + sb] : 0.0f;
        if (gJs) {
            ca *= sa < S ? gsc * w[sa] : 0.0f;
            cb *= sb < S ? gsc * w[sb] : 0.0f;
        }
        uint4 o;
        tf32_split(ca, o.x, o.z);
        tf32_split(cb, o.y, o.w);
        s_c[u] = o;
    }
    const float c1 = E.pf * E.rf, pcm = E.pcf + E.mcf, mcn = -E.mcf;
    const uint32_t one = __float_as_uint(1.0f);
    for (int k = 0; k < ntiles; k++) {
        if (k + kAdjStages - 1 < ntiles) issue(k + kAdjStages - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group %0;" ::"n"(kAdjStages - 1) : "memory");  // tile k has landed
        __syncthreads();
        const int st = k % kAdjStages, b0 = b_lo + k * kAdjBT, nb = min(kAdjBT, b_hi - b0);
        const float *sg = s_g + (size_t)st * kAdjBT * L.RS;
        const uint32_t *sm_m = s_m + st * kAdjBT;
        if (want_g)
            for (int j = tid; j < nb; j += nth) {  // m_b c1 D_b, D_b = sum_t d_t x[b][t]
                float D = 0.0f;
                if (xst) {
                    const float *xr = s_x + ((size_t)st * kAdjBT + j) * L.XS;
                    for (int t = 0; t < T; t++) D = fmaf(s_d[t], xr[t], D);
                } else {
                    const float *xr = x + (size_t)(b0 + j) * T;
                    for (int t = 0; t < T; t++) D = fmaf(s_d[t], __ldg(xr + t), D);
                }
                s_D[j] = (float)sm_m[j] * c1 * D;
            }
        // warp w: the M tile of blocks 16 (w mod 4) .. + 15, K steps of parity w / 4
        const int mb = 16 * (warp % (kAdjBT / 16)), kh = warp / (kAdjBT / 16);
        float acc[TT / 8][4];
#pragma unroll
        for (int n = 0; n < TT / 8; n++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[n][q] = 0.0f;
        float u0 = 0.0f, u1 = 0.0f;  // blocks mb + gid and mb + gid + 8
        if (mb < nb) {
            const float *r0 = sg + (size_t)(mb + gid) * L.RS, *r1 = r0 + 8 * L.RS;
            for (int k8 = 8 * kh; k8 < L.K8; k8 += 8 * kAdjKSplit) {
                const int sa = k8 + tig, sb = sa + 4;
                // A[m][k]: m = gid (+8), k = tig (+4)
                const float gv[4] = {r0[sa], r1[sa], r0[sb], r1[sb]};
                const float wa = s_w[sa], wb = s_w[sb];
                uint32_t a[4];
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    bool ore;
                    if (ROWS) {
                        const float *rw = (e & 1) ? r1 : r0;
                        const int s = (e & 2) ? sb : sa;
                        ore = (__float_as_uint(rw[L.K8 + (s >> 5)]) >> (s & 31)) & 1u;
                        v[e] = gv[e];
                    } else {
                        ore = THR ? gv[e] >= E.g_thr : relax_ore(gv[e], E);
                        v[e] = ore ? fmaf(gv[e], c1, -pcm) : mcn;
                    }
                    a[e] = ore ? one : 0u;
                }
                u0 = fmaf(wb, v[2], fmaf(wa, v[0], u0));
                u1 = fmaf(wb, v[3], fmaf(wa, v[1], u1));
                const uint4 *cb = s_c + ((k8 >> 3) * TT + gid) * 4 + tig;
#pragma unroll
                for (int n = 0; n < TT / 8; n++) {
                    const uint4 p = cb[32 * n];  // B[k][n]: k = tig (+4), n = gid
                    const uint32_t bh[2] = {p.x, p.y}, bl[2] = {p.z, p.w};
                    mma_tf32(acc[n], a, bh);
                    mma_tf32(acc[n], a, bl);
                }
            }
        }
        // the odd-K warps hand their sums to the even-K warp of their M tile
        float *xch = s_x2 + ((size_t)(warp % (kAdjBT / 16)) * 32 + lane) * (TT / 2 + 2);
        if (kh == 1) {
#pragma unroll
            for (int n = 0; n < TT / 8; n++)
#pragma unroll
                for (int q = 0; q < 4; q++) xch[4 * n + q] = acc[n][q];
            xch[TT / 2] = u0;
            xch[TT / 2 + 1] = u1;
        }
        __syncthreads();
        if (kh == 0 && mb < nb) {
#pragma unroll
            for (int n = 0; n < TT / 8; n++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[n][q] += xch[4 * n + q];
            u0 += xch[TT / 2];
            u1 += xch[TT / 2 + 1];
            u0 += __shfl_xor_sync(0xffffffffu, u0, 1);
            u0 += __shfl_xor_sync(0xffffffffu, u0, 2);
            u1 += __shfl_xor_sync(0xffffffffu, u1, 1);
            u1 += __shfl_xor_sync(0xffffffffu, u1, 2);
            // D[m][n] at m = gid (+8 for q >= 2), n = 2 tig + (q & 1)
#pragma unroll
            for (int n = 0; n < TT / 8; n++)
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int j = mb + gid + (q >= 2 ? 8 : 0), t = 8 * n + 2 * tig + (q & 1);
                    if (j < nb && t < nt) {
                        const float mj = (float)sm_m[j], uj = q >= 2 ? u1 : u0;
                        const float val = ROWS ? uj - mj * acc[n][q] : mj * (uj - acc[n][q]);
                        gx[(size_t)(b0 + j) * T + t0 + t] = s_d[t0 + t] * val;
                    }
                }
        }
        if (want_g) {
            __syncthreads();  // s_D
            // the tile's rows of dJ/dg are one contiguous stretch: consecutive
            // threads write consecutive 16-byte chunks (streaming stores)
            float *out = gg + (size_t)b0 * S;
            if (gvec) {
                const int cpr = S / 4;
                for (int i = tid; i < nb * cpr; i += nth) {
                    const int j = (int)fdiv((uint32_t)i, cmag), q = i - j * cpr;
                    const float f = s_D[j];
                    const float *row = sg + (size_t)j * L.RS;
                    const float4 g4 = *reinterpret_cast<const float4 *>(row + 4 * q);
                    const float4 w4 = *reinterpret_cast<const float4 *>(s_w + 4 * q);
                    const float gs[4] = {g4.x, g4.y, g4.z, g4.w}, ws[4] = {w4.x, w4.y, w4.z, w4.w};
                    float o4[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int sc = 4 * q + e;
                        const bool ore = ROWS ? ((__float_as_uint(row[L.K8 + (sc >> 5)]) >> (sc & 31)) & 1u)
                                              : (THR ? gs[e] >= E.g_thr : relax_ore(gs[e], E));
                        o4[e] = ore ? ws[e] * f : 0.0f;
                    }
                    __stcs(reinterpret_cast<float4 *>(out + (size_t)j * S + 4 * q), make_float4(o4[0], o4[1], o4[2], o4[3]));
                }
            } else {
                for (int i = tid; i < nb * S; i += nth) {
                    const int j = (int)fdiv((uint32_t)i, smag), sc = i - j * S;
                    const float *row = sg + (size_t)j * L.RS;
                    const bool ore = ROWS ? ((__float_as_uint(row[L.K8 + (sc >> 5)]) >> (sc & 31)) & 1u)
                                          : (THR ? row[sc] >= E.g_thr : relax_ore(row[sc], E));
                    __stcs(out + i, ore ? s_w[sc] * s_D[j] : 0.0f);
                }
            }
        }
        __syncthreads();  // the stage is refilled next
    }
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
    const RelaxEcon E = relax_econ(m, beta, m_ref);
    const RelaxRows Rw{m->val, m->R, m->ore_off};
    // block ranges: one forward CTA per SM over the scenario tiles, whole
    // 32-block tiles each
    const int nr = relax_fwd_ctas(m, B, S);
    const size_t TS = (size_t)T * S;
    // the adjoint's coefficients: P_t'(O) [T][S], then w_s / gJ [S]
    if (m->relax_coef_floats < TS + S) {
        cudaFree(m->relax_coef);
        m->relax_coef = nullptr;
        m->relax_coef_floats = 0;
        m->rc_npv = m->rc_ore = nullptr;
        MM_CUDA_TRY(cudaMalloc(&m->relax_coef, (TS + S) * sizeof(float)), "allocate relaxed coefficients");
        m->relax_coef_floats = TS + S;
    }
    m->rc_npv = m->rc_ore = nullptr;  // valid again once the finish is launched
    // scratch: range partials of O and V (FP32), then the terms (FP64)
    const int nchunk = (S + 31) / 32;
    st = relax_scratch(m, 2 * (size_t)nr * TS + 2 * TS);
    if (st != MM_OK) return st;
    float *part_o = m->relax_scratch, *part_v = part_o + (size_t)nr * TS;
    double *term = reinterpret_cast<double *>(part_v + (size_t)nr * TS);
    const int stall = m->test_stall_relax;  // test-only, one-shot
    m->test_stall_relax = 0;
    st = g_dev ? relax_fwd_launch<float>(m, x_dev, g_dev, Rw, m->mass, B, S, T, E, part_o, part_v, nr, m->stream, stall)
               : relax_fwd_launch<double>(m, x_dev, m->grade, Rw, m->mass, B, S, T, E, part_o, part_v, nr, m->stream,
                                          stall);
    if (st != MM_OK) return st;
    // the finish launches as a programmatic dependent of the forward grid, so
    // its launch overlaps the forward's tail
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nchunk, (unsigned)T);
    cfg.blockDim = dim3(32 * kFinWarps);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = m->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MM_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_relax_finish, (const float *)part_o, (const float *)part_v, (int32_t)nr,
                                   (int32_t)S, (int32_t)T, (const double *)m->disc, (const uint64_t *)m->target, E,
                                   ore_t_dev, term, m->relax_tick, npv_dev, J_dev, m->relax_coef,
                                   m->relax_coef + TS),
                "k_relax_finish launch");
    m->rc_npv = npv_dev;
    m->rc_ore = ore_t_dev;
    m->rc_beta = beta;
    m->rc_mref = m_ref;
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
    const RelaxEcon E = relax_econ(m, beta, m_ref);
    const RelaxRows Rw{m->val, m->R, m->ore_off};
    const bool rows = g_dev == nullptr;
    // the tensor-core adjoint, period tiles of up to kAdjMaxTT, when its shared memory fits
    size_t need = 0;
    for (int tb = 0; tb < T; tb += kAdjMaxTT) {
        const int tt = (std::min(kAdjMaxTT, T - tb) + 7) / 8 * 8;
        need = std::max(need, adj_layout(S, T, tt, rows, gg_dev && tb == 0 && T <= kAdjMaxTT).floats * sizeof(float));
    }
    const bool tc = need + 1024 <= (size_t)m->max_smem_optin;
    // the last forward's outputs with the same smoothing: its coefficients
    // are reused (scaled by gJ in the adjoint), no coefficient launch
    const bool cached = tc && m->relax_coef && npv_dev == m->rc_npv && ore_t_dev == m->rc_ore &&
                        beta == m->rc_beta && m_ref == m->rc_mref;
    const float *w = nullptr, *c = nullptr;
    int cs = Sp;
    if (cached) {
        c = m->relax_coef;
        w = m->relax_coef + (size_t)T * S;
        cs = S;
    } else {
        st = relax_scratch(m, (size_t)S + (size_t)T * Sp);
        if (st != MM_OK) return st;
        float *ws = m->relax_scratch, *cw = ws + S;
        // small CTAs: each forms the scenario mean and std itself, so more SMs
        // share the FP64 work
        k_relax_coef<<<(unsigned)(((size_t)T * S + 127) / 128), 128, 0, m->stream>>>(npv_dev, ore_t_dev, m->target,
                                                                                      gJ_dev, S, T, Sp, E, ws, cw);
        st = check_launch("k_relax_coef");
        if (st != MM_OK) return st;
        w = ws;
        c = cw;
    }
    if (tc) {
        const int vec = (!rows && S % 4 == 0 && ((uintptr_t)g_dev & 15u) == 0) ? 1 : 0;
        const int xvec = (T % 4 == 0 && ((uintptr_t)x_dev & 15u) == 0) ? 1 : 0;
        const int gvec = (gg_dev && S % 4 == 0 && ((uintptr_t)gg_dev & 15u) == 0) ? 1 : 0;
        const float *gf = rows ? nullptr : g_dev;
        for (int tb = 0; tb < T; tb += kAdjMaxTT) {
            const int tt = (std::min(kAdjMaxTT, T - tb) + 7) / 8 * 8;
            const size_t sm = adj_layout(S, T, tt, rows, gg_dev && tb == 0 && T <= kAdjMaxTT).floats * sizeof(float);
            const void *fn = nullptr;
            switch (tt) {
#define MM_ADJ_FN(V)                                                                                               \
    rows ? (E.use_thr ? (const void *)k_relax_adj_tc<double, V, true> : (const void *)k_relax_adj_tc<double, V, false>) \
         : (E.use_thr ? (const void *)k_relax_adj_tc<float, V, true> : (const void *)k_relax_adj_tc<float, V, false>)
                case 8: fn = MM_ADJ_FN(8); break;
                case 16: fn = MM_ADJ_FN(16); break;
                case 24: fn = MM_ADJ_FN(24); break;
                default: fn = MM_ADJ_FN(32); break;
#undef MM_ADJ_FN
            }
            MM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm), "adjoint smem");
            int per_sm = 1;
            MM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * kAdjWarps, sm), "occupancy");
            const int grid = std::max(1, std::min((B + 15) / 16, std::max(1, per_sm) * m->num_sms));
            // a programmatic dependent of the previous launch (the coefficients,
            // or the previous period tile): its first copies overlap that launch's tail
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)grid);
            cfg.blockDim = dim3(32 * kAdjWarps);
            cfg.dynamicSmemBytes = sm;
            cfg.stream = m->stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const void *gp = rows ? (const void *)m->grade : (const void *)gf;
            int32_t Sp32 = cs, tb32 = tb;
            const double *gJs = cached ? gJ_dev : nullptr;
            void *args[] = {(void *)&x_dev, (void *)&gp, (void *)&Rw, (void *)&m->mass, (void *)&w, (void *)&c,
                            (void *)&Sp32, (void *)&gJs, (void *)&m->disc, (void *)&B, (void *)&S, (void *)&T, (void *)&tb32,
                            (void *)&E, (void *)&vec, (void *)&xvec, (void *)&gvec, (void *)&gx_dev, (void *)&gg_dev};
            MM_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, args), "adjoint launch");
            st = check_launch("k_relax_adj_tc");
            if (st != MM_OK) return st;
        }
        return MM_OK;
    }
    // the one-warp-per-block kernel for rows that do not fit the staged tiles
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
