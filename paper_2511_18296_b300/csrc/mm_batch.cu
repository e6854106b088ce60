// Batched multi-chain evaluation: many independent search chains (each its own
// block model, scenario count and move batch) evaluated in ONE persistent
// launch fed by a device work queue.
//
// The queue is a list of items (chain, range of that chain's moves), ordered
// largest estimated cost first.  Every CTA of the persistent grid takes the next
// item with one atomicAdd (drawn together with its previous item's ticket), stages the chain's small tables in shared memory,
// evaluates the range with the same per-warp evaluator as the single-model
// path (its compile-time-shaped form where the chain's scenario count has one,
// the run-time-shaped form otherwise), and publishes the range's 32 best keys.
// The CTA that completes a chain's last item (a ticket counter per chain: no
// CTA ever waits for another) merges that chain's lists into its top k and,
// when asked, applies the chain's best move with the single-model apply code.
// Nothing in the launch allocates or synchronises with the host, so a run can
// be captured into a CUDA graph; the tile shape (moves per item, CTAs per SM)
// and each scenario class's team width and prefetch distance are chosen by
// mm_batch_autotune.
#include <algorithm>
#include <vector>

#include "mm_eval_tiled.cuh"

namespace mm {

ApplyArgs apply_args(mm_model *m);
int default_team(int S);

// Evaluator shapes compiled into the batched kernel.  A chain always runs with
// the team width of the single-model path (default_team(S)), so its sums are
// formed in the same order and its results are the same bits; the
// compile-time-shaped forms cover the common scenario counts, the run-time
// shaped form of the same team width covers every other S.
enum BatchVariant : int32_t {
    kBvG4 = 0,     // run-time shaped, 4-lane teams, up to 4 quads per lane (S <= 64)
    kBvG8 = 1,     // 8-lane teams (S <= 128)
    kBvG16 = 2,    // 16-lane teams (S <= 256)
    kBvG32 = 3,    // 32-lane teams, up to 8 quads (S <= 1024)
    kBvT4K1 = 4,   // compile-time shaped: 4-lane teams, 1 quad per lane (S = 16)
    kBvT4K2 = 5,   // 4-lane teams, 2 quads (S = 32)
    kBvT4K3 = 6,   // 4-lane teams, 3 quads (S = 48)
    kBvT4K4 = 7,   // 4-lane teams, 4 quads (S = 64)
    kBvT8K3T = 8,  // 8-lane teams, 3 quads + a tail quad (S = 100 .. 124, S % 4 == 0)
};

// One chain as the kernel sees it.
struct ChainDev {
    EvalArgs E;    // evaluator arguments of the chain's model and buffers
    ApplyArgs AP;  // apply arguments of the chain's model
    int32_t variant;
    int32_t list0;    // first of the chain's published lists
    int32_t n_items;  // items (and lists) of the chain
    int32_t k;
    int32_t do_apply;
    int32_t *idx_out;
    float *top_out;
    int32_t *count_out;
};

struct BatchItem {
    int32_t chain;
    int32_t item;  // index among the chain's items (its list slot)
    int64_t r0, r1;
};

struct BatchArgs {
    const ChainDev *chains;
    const BatchItem *items;
    int32_t n_items;
    uint32_t *next;   // [0] queue head; [1 + c] items completed of chain c
    uint64_t *lists;  // [total items][32]
};

constexpr int kBatchMaxT = 64;  // chains with more periods are not batched (tables staged per item)

// The CTA's current item: its chain's evaluator arguments and small tables,
// and the evaluator's per-warp lists.  At namespace scope so that each
// evaluator shape below, a separate (not inlined) function, addresses them as
// shared memory.
__shared__ EvalShared b_sh;
__shared__ __align__(16) EvalArgs b_A;
__shared__ float b_dd[(kBatchMaxT + 1) * (kBatchMaxT + 1)];
__shared__ int64_t b_mined[kBatchMaxT + 1];
__shared__ uint64_t b_cap[kBatchMaxT + 1];

// One evaluator shape over the calling warp's moves [r0, r1) of the current
// item; returns the warp's top-32 keys.  Not inlined: compiled together, the
// nine shapes need more registers than the kernel's occupancy allows, and
// each alone needs fewer.
template <int TEAM, int QMAX, int KF, bool TAIL>
static __device__ __noinline__ uint64_t batch_range(int64_t r0, int64_t r1) {
    uint64_t wtk = 0;
    eval_warp_range<TEAM, QMAX, false, false, KF, TAIL, true>(b_A, b_sh, b_A.tab, b_dd, b_mined, b_cap, r0, r1, wtk);
    return wtk;
}

__global__ void __launch_bounds__(kEvalThreads, MM_EVAL_MINB) k_batch_eval(BatchArgs B) {
    constexpr int NW = kEvalThreads / 32;
    EvalArgs &sA = b_A;
    float *s_dd = b_dd;
    int64_t *s_mined = b_mined;
    uint64_t *s_cap = b_cap;
    __shared__ uint64_t s_wl[NW][32];
    __shared__ __align__(16) float s_apply_tab[kApplyTabMax];
    __shared__ int s_item, s_last, s_best;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_item = (int)atomicAdd(B.next, 1u);
    __syncthreads();
    int it = s_item;
    for (;;) {
        if (it >= B.n_items) break;
        const BatchItem I = B.items[it];
        const ChainDev *C = B.chains + I.chain;
        // the chain's evaluator arguments and small tables into shared memory
        {
            const int *src = reinterpret_cast<const int *>(&C->E);
            int *dst = reinterpret_cast<int *>(&sA);
            for (int i = tid; i < (int)(sizeof(EvalArgs) / sizeof(int)); i += kEvalThreads) dst[i] = __ldg(src + i);
        }
        __syncthreads();
        const int T1 = sA.T + 1;
        for (int i = tid; i < T1 * T1; i += kEvalThreads) s_dd[i] = __ldg(sA.ddt + i);
        for (int i = tid; i < T1; i += kEvalThreads) {
            s_mined[i] = sA.minedT[i];
            s_cap[i] = sA.cap[i];
        }
        __syncthreads();
        // this warp's share of the item's moves
        const int64_t len = I.r1 - I.r0;
        const int64_t r0 = I.r0 + warp * len / NW, r1 = I.r0 + (warp + 1) * len / NW;
        uint64_t wtk;
        switch (C->variant) {
            case kBvT4K1: wtk = batch_range<4, 1, 1, false>(r0, r1); break;
            case kBvT4K2: wtk = batch_range<4, 1, 2, false>(r0, r1); break;
            case kBvT4K3: wtk = batch_range<4, 1, 3, false>(r0, r1); break;
            case kBvT4K4: wtk = batch_range<4, 1, 4, false>(r0, r1); break;
            case kBvT8K3T: wtk = batch_range<8, 1, 3, true>(r0, r1); break;
            case kBvG4: wtk = batch_range<4, 4, 0, false>(r0, r1); break;
            case kBvG8: wtk = batch_range<8, 4, 0, false>(r0, r1); break;
            case kBvG16: wtk = batch_range<16, 4, 0, false>(r0, r1); break;
            default: wtk = batch_range<32, 8, 0, false>(r0, r1); break;
        }
        const int32_t list0 = C->list0, n_items = C->n_items;
        step_publish(B.lists + (size_t)(list0 + I.item) * 32, wtk);
        // ticket: the CTA completing the chain's last item finishes the chain
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            s_last = atomicAdd(B.next + 1 + I.chain, 1u) == (uint32_t)(n_items - 1);
            s_item = (int)atomicAdd(B.next, 1u);  // the next item, drawn beside the ticket
        }
        __syncthreads();
        const int next = s_item;
        if (s_last) {
            __threadfence();
            const uint64_t t = block_merge_lists<NW>(B.lists + (size_t)list0 * 32, n_items, s_wl);
            if (warp == 0) {
                const int best = warp_write_topk(t, C->k, sA.n, sA.status, C->idx_out, C->top_out,
                                                 C->count_out);
                if (lane == 0) s_best = best;
            }
            __syncthreads();
            if (C->do_apply) {
                const int b = s_best;
                const int2 mv = b >= 0 ? __ldg(sA.moves + b) : make_int2(0, -1);
                apply_block(C->AP, mv, b >= 0 ? 1 : 0, s_apply_tab);
            }
        }
        __syncthreads();  // shared state is reused by the next item
        it = next;
    }
}

}  // namespace mm

using namespace mm;

struct mm_batch {
    int n_chains = 0;
    int k = 0;
    int do_apply = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int max_per_sm = 1;               // occupancy of k_batch_eval
    int moves_per_item = 2048;        // tile shape: moves per queue item
    int ctas_per_sm = 0;              // 0 = max_per_sm
    std::vector<ChainDev> chains;     // host copy (list0 / n_items follow the tile shape)
    std::vector<mm_model *> models;   // each chain's model
    std::vector<int64_t> n_moves;
    std::vector<int> S;
    std::vector<int> team;            // each chain's team width (lanes per move)
    ChainDev *d_chains = nullptr;
    BatchItem *d_items = nullptr;
    int n_items = 0, items_cap = 0;
    uint32_t *d_next = nullptr;       // [1 + n_chains]
    uint64_t *d_lists = nullptr;      // [items_cap][32]
    int lists_cap = 0;
};

// Largest quads per lane of a team width's run-time shaped form.
static int team_qmax(int team) { return team == 32 ? 8 : 4; }

static bool team_fits(int S, int team) {
    const int nq = (S + 3) / 4;
    return (team == 4 || team == 8 || team == 16 || team == 32) && (nq + team - 1) / team <= team_qmax(team);
}

static int batch_variant(const mm_model *m, int team) {
    const int generic = team == 4 ? kBvG4 : team == 8 ? kBvG8 : team == 16 ? kBvG16 : kBvG32;
    if (m->S % 4 != 0 || !m->ctab) return generic;
    const int nq = m->S / 4;
    const int kf = nq / team;
    const bool tail = nq % team != 0;
    if (team == 4 && !tail && kf >= 1 && kf <= 4) return kBvT4K1 + (kf - 1);
    if (team == 8 && tail && kf == 3) return kBvT8K3T;
    return generic;
}

// Queue items for the current tile shape, largest estimated cost first, and
// the chains' list offsets; uploads both (synchronous: not called during runs).
static mm_status batch_build(mm_batch *b) {
    std::vector<BatchItem> items;
    int list0 = 0;
    for (int c = 0; c < b->n_chains; c++) {
        const int64_t n = b->n_moves[c];
        const int per = b->moves_per_item;
        const int ni = n > 0 ? (int)((n + per - 1) / per) : 0;
        b->chains[c].list0 = list0;
        b->chains[c].n_items = ni;
        for (int i = 0; i < ni; i++) {
            const int64_t r0 = (int64_t)i * per, r1 = std::min<int64_t>(n, r0 + per);
            items.push_back(BatchItem{c, i, r0, r1});
        }
        list0 += ni;
    }
    // longest processing time first: (moves) x (scenarios, plus decode work)
    std::stable_sort(items.begin(), items.end(), [&](const BatchItem &x, const BatchItem &y) {
        const double cx = (double)(x.r1 - x.r0) * (b->S[x.chain] + 16);
        const double cy = (double)(y.r1 - y.r0) * (b->S[y.chain] + 16);
        return cx > cy;
    });
    b->n_items = (int)items.size();
    if (b->n_items > b->items_cap) {
        cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        MM_CUDA_TRY(cudaMalloc(&b->d_items, sizeof(BatchItem) * (size_t)b->n_items), "allocate batch queue");
        b->items_cap = b->n_items;
    }
    if (list0 > b->lists_cap) {
        cudaFree(b->d_lists);
        b->d_lists = nullptr;
        b->lists_cap = 0;
        MM_CUDA_TRY(cudaMalloc(&b->d_lists, sizeof(uint64_t) * 32 * (size_t)list0), "allocate batch lists");
        b->lists_cap = list0;
    }
    if (b->n_items > 0)
        MM_CUDA_TRY(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice),
                    "upload batch queue");
    MM_CUDA_TRY(cudaMemcpy(b->d_chains, b->chains.data(), sizeof(ChainDev) * b->chains.size(), cudaMemcpyHostToDevice),
                "upload chain descriptors");
    return MM_OK;
}

static void batch_free(mm_batch *b) {
    if (!b) return;
    cudaFree(b->d_chains);
    cudaFree(b->d_items);
    cudaFree(b->d_next);
    cudaFree(b->d_lists);
    delete b;
}

extern "C" {

mm_status mm_batch_create(const mm_chain *chains, int32_t n_chains, int32_t k, int32_t apply, void *cuda_stream,
                          mm_batch **out) {
    if (!out) return set_error(MM_ERR_INVALID_ARG, "NULL output handle");
    *out = nullptr;
    if (!chains || n_chains < 1) return set_error(MM_ERR_INVALID_ARG, "need at least one chain");
    if (k < 1 || k > 32) return set_error(MM_ERR_INVALID_ARG, "batched top-k: k = %d outside 1..32", k);
    for (int c = 0; c < n_chains; c++) {
        const mm_chain &ch = chains[c];
        mm_model *m = ch.model;
        if (!m) return set_error(MM_ERR_INVALID_ARG, "chain %d: NULL model", c);
        if (!m->has_schedule) return set_error(MM_ERR_STATE, "chain %d: no schedule installed", c);
        if (!m->uniform_mass) return set_error(MM_ERR_INVALID_ARG, "chain %d: batched evaluation needs equal block masses", c);
        if (m->sig) return set_error(MM_ERR_INVALID_ARG, "chain %d: batched evaluation does not take uncertainty weights", c);
        if (m->T > kBatchMaxT) return set_error(MM_ERR_INVALID_ARG, "chain %d: T = %d > %d", c, m->T, kBatchMaxT);
        if (ch.n_moves < 0 || ch.n_moves > 0x7fffffffLL)
            return set_error(MM_ERR_INVALID_ARG, "chain %d: move count out of range", c);
        if (ch.n_moves > 0 && (!ch.moves_dev || !ch.score_dev || !ch.feasible_dev))
            return set_error(MM_ERR_INVALID_ARG, "chain %d: NULL move or output buffer", c);
        if (((uintptr_t)ch.moves_dev & 7u) != 0) return set_error(MM_ERR_INVALID_ARG, "chain %d: moves not 8-byte aligned", c);
        if (!ch.idx_dev || !ch.topscore_dev || !ch.count_dev)
            return set_error(MM_ERR_INVALID_ARG, "chain %d: NULL top-k output", c);
        if (apply && m->S > kEvalThreads)
            return set_error(MM_ERR_INVALID_ARG, "chain %d: apply in the batch needs S <= %d", c, kEvalThreads);
        for (int d = 0; d < c; d++)
            if (chains[d].model == m) return set_error(MM_ERR_INVALID_ARG, "chains %d and %d share a model", d, c);
    }
    mm_batch *b = new mm_batch();
    b->n_chains = n_chains;
    b->k = k;
    b->do_apply = apply ? 1 : 0;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->num_sms = chains[0].model->num_sms;
    b->chains.resize(n_chains);
    b->models.resize(n_chains);
    b->n_moves.resize(n_chains);
    b->S.resize(n_chains);
    for (int c = 0; c < n_chains; c++) {
        const mm_chain &ch = chains[c];
        mm_model *m = ch.model;
        ChainDev &d = b->chains[c];
        memset(&d, 0, sizeof(d));
        d.E = eval_args(m, ch.moves_dev, ch.n_moves, ch.score_dev, ch.feasible_dev, nullptr, nullptr);
        const int team = default_team(m->S);
        d.variant = batch_variant(m, team);
        const int nq = (m->S + 3) / 4;
        d.E.qpl = (nq + team - 1) / team;  // quads per lane of the run-time shaped forms
        d.E.prefetch = 0;
        b->team.push_back(team);
        d.AP = apply_args(m);
        d.k = k;
        d.do_apply = b->do_apply;
        d.idx_out = ch.idx_dev;
        d.top_out = ch.topscore_dev;
        d.count_out = ch.count_dev;
        b->n_moves[c] = ch.n_moves;
        b->S[c] = m->S;
        b->models[c] = m;
    }
    cudaError_t e = cudaMalloc(&b->d_chains, sizeof(ChainDev) * (size_t)n_chains);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(uint32_t) * (size_t)(n_chains + 1));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->max_per_sm, k_batch_eval, kEvalThreads, 0);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_status(e, "create batch");
    }
    if (b->max_per_sm < 1) b->max_per_sm = 1;
    mm_status st = batch_build(b);
    if (st != MM_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return MM_OK;
}

void mm_batch_destroy(mm_batch *b) { batch_free(b); }

mm_status mm_batch_set_tile(mm_batch *b, int32_t moves_per_item, int32_t ctas_per_sm) {
    if (!b) return set_error(MM_ERR_INVALID_ARG, "NULL batch");
    if (moves_per_item < 64 || moves_per_item > (1 << 20) || (moves_per_item & 63) != 0)
        return set_error(MM_ERR_INVALID_ARG, "moves_per_item must be a multiple of 64 in 64..1048576");
    if (ctas_per_sm < 0 || ctas_per_sm > b->max_per_sm)
        return set_error(MM_ERR_INVALID_ARG, "ctas_per_sm must be 0..%d", b->max_per_sm);
    b->moves_per_item = moves_per_item;
    b->ctas_per_sm = ctas_per_sm;
    return batch_build(b);
}

mm_status mm_batch_set_chain(mm_batch *b, int32_t chain, int32_t team, int32_t prefetch) {
    if (!b) return set_error(MM_ERR_INVALID_ARG, "NULL batch");
    if (chain < 0 || chain >= b->n_chains) return set_error(MM_ERR_INVALID_ARG, "chain %d outside 0..%d", chain, b->n_chains - 1);
    const int S = b->S[chain];
    if (team == 0) team = default_team(S);
    if (!team_fits(S, team))
        return set_error(MM_ERR_INVALID_ARG, "chain %d: team width %d does not fit S = %d", chain, team, S);
    if (prefetch < -1 || prefetch > 8) return set_error(MM_ERR_INVALID_ARG, "prefetch must be -1..8");
    ChainDev &d = b->chains[chain];
    d.variant = batch_variant(b->models[chain], team);
    d.E.qpl = ((S + 3) / 4 + team - 1) / team;
    d.E.prefetch = prefetch < 0 ? 0 : prefetch;
    b->team[chain] = team;
    MM_CUDA_TRY(cudaMemcpy(b->d_chains + chain, &d, sizeof(ChainDev), cudaMemcpyHostToDevice), "upload chain descriptor");
    return MM_OK;
}

mm_status mm_batch_get_chain(const mm_batch *b, int32_t chain, int32_t *team, int32_t *prefetch) {
    if (!b) return set_error(MM_ERR_INVALID_ARG, "NULL batch");
    if (chain < 0 || chain >= b->n_chains) return set_error(MM_ERR_INVALID_ARG, "chain %d outside 0..%d", chain, b->n_chains - 1);
    if (team) *team = b->team[chain];
    if (prefetch) *prefetch = b->chains[chain].E.prefetch;
    return MM_OK;
}

mm_status mm_batch_get_tile(const mm_batch *b, int32_t *moves_per_item, int32_t *ctas_per_sm, int32_t *n_items) {
    if (!b) return set_error(MM_ERR_INVALID_ARG, "NULL batch");
    if (moves_per_item) *moves_per_item = b->moves_per_item;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm > 0 ? b->ctas_per_sm : b->max_per_sm;
    if (n_items) *n_items = b->n_items;
    return MM_OK;
}

mm_status mm_batch_run(mm_batch *b) {
    if (!b) return set_error(MM_ERR_INVALID_ARG, "NULL batch");
    MM_CUDA_TRY(cudaMemsetAsync(b->d_next, 0, sizeof(uint32_t) * (size_t)(b->n_chains + 1), b->stream),
                "reset batch queue");
    // chains without moves: empty top-k (and no apply) without a queue item
    for (int c = 0; c < b->n_chains; c++)
        if (b->n_moves[c] == 0)
            MM_CUDA_TRY(cudaMemsetAsync(b->chains[c].count_out, 0, sizeof(int32_t), b->stream), "clear count");
    // an apply in the batch updates the FP64 totals: any update a fused step
    // left due on a chain's model is done first, on the batch's stream
    if (b->do_apply)
        for (mm_model *m : b->models) {
            const mm_status st = settle_money(m, b->stream);
            if (st != MM_OK) return st;
        }
    if (b->n_items == 0) return MM_OK;
    const int per_sm = b->ctas_per_sm > 0 ? b->ctas_per_sm : b->max_per_sm;
    const int grid = std::min(b->n_items, b->num_sms * per_sm);
    BatchArgs A;
    A.chains = b->d_chains;
    A.items = b->d_items;
    A.n_items = b->n_items;
    A.next = b->d_next;
    A.lists = b->d_lists;
    k_batch_eval<<<grid, kEvalThreads, 0, b->stream>>>(A);
    return check_launch("k_batch_eval");
}

// Mean time of `reps` runs (after one warm-up run) with CUDA events on the
// batch's stream.
static mm_status batch_time(mm_batch *b, int reps, cudaEvent_t e0, cudaEvent_t e1, float *ms_out) {
    mm_status st = mm_batch_run(b);  // warm-up
    float tot = 0.0f;
    for (int r = 0; r < reps && st == MM_OK; r++) {
        float ms = 0.0f;
        cudaEventRecord(e0, b->stream);
        st = mm_batch_run(b);
        cudaEventRecord(e1, b->stream);
        cudaError_t se = cudaEventSynchronize(e1);
        if (se == cudaSuccess) se = cudaEventElapsedTime(&ms, e0, e1);
        if (se != cudaSuccess && st == MM_OK) st = cuda_status(se, "time a batch run");
        tot += ms;
    }
    *ms_out = tot / (float)reps;
    return st;
}

mm_status mm_batch_autotune(mm_batch *b, int32_t reps, int32_t *moves_per_item, int32_t *ctas_per_sm,
                            float *best_ms) {
    if (!b) return set_error(MM_ERR_INVALID_ARG, "NULL batch");
    if (reps < 1) reps = 1;
    if (b->do_apply) return set_error(MM_ERR_STATE, "autotune a batch created without apply (runs change no state)");
    const int tiles[] = {512, 1024, 2048, 4096, 8192, 16384};
    std::vector<int> ctas = {0};
    if (b->max_per_sm > 1) ctas.push_back(b->max_per_sm - 1);
    cudaEvent_t e0, e1;
    MM_CUDA_TRY(cudaEventCreate(&e0), "create event");
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_status(ce, "create event");
    }
    float best = 1e30f;
    int best_tile = b->moves_per_item, best_ctas = b->ctas_per_sm;
    mm_status st = MM_OK;
    // 1. tile shape: moves per item x CTAs per SM
    for (int tile : tiles) {
        for (int cp : ctas) {
            b->moves_per_item = tile;
            b->ctas_per_sm = cp;
            float ms = 0.0f;
            if ((st = batch_build(b)) != MM_OK) break;
            if ((st = batch_time(b, reps, e0, e1, &ms)) != MM_OK) break;
            if (ms < best) {
                best = ms;
                best_tile = tile;
                best_ctas = cp;
            }
        }
        if (st != MM_OK) break;
    }
    if (st == MM_OK) {
        b->moves_per_item = best_tile;
        b->ctas_per_sm = best_ctas;
        st = batch_build(b);
    }
    // 2. team width per scenario class (chains with the same S): every width
    //    that fits, the class's other chains unchanged; a width is kept only
    //    if it beats the best time so far by more than 1 %
    std::vector<int> classes(b->S.begin(), b->S.end());
    std::sort(classes.begin(), classes.end());
    classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
    for (int S : classes) {
        if (st != MM_OK) break;
        int keep = -1;
        for (int c = 0; c < b->n_chains; c++)
            if (b->S[c] == S) keep = b->team[c];
        for (int team = 4; team <= 32 && st == MM_OK; team *= 2) {
            if (team == keep || !team_fits(S, team)) continue;
            for (int c = 0; c < b->n_chains && st == MM_OK; c++)
                if (b->S[c] == S) st = mm_batch_set_chain(b, c, team, b->chains[c].E.prefetch);
            float ms = 0.0f;
            if (st == MM_OK) st = batch_time(b, reps, e0, e1, &ms);
            if (st == MM_OK && ms < best * 0.99f) {
                best = ms;
                keep = team;
            }
        }
        for (int c = 0; c < b->n_chains && st == MM_OK; c++)
            if (b->S[c] == S) st = mm_batch_set_chain(b, c, keep, b->chains[c].E.prefetch);
    }
    // 3. L1 prefetch distance (evaluation batches ahead) per scenario class,
    //    the other classes unchanged: a class whose rows stay in L2 loses by
    //    prefetching, one whose rows come from DRAM may gain; kept only if it
    //    beats the best time so far by more than 1 %
    for (int S : classes) {
        if (st != MM_OK) break;
        int keep = -1;
        for (int c = 0; c < b->n_chains; c++)
            if (b->S[c] == S) keep = b->chains[c].E.prefetch;
        for (int pf = 0; pf <= 2 && st == MM_OK; pf++) {
            if (pf == keep) continue;
            for (int c = 0; c < b->n_chains && st == MM_OK; c++)
                if (b->S[c] == S) st = mm_batch_set_chain(b, c, b->team[c], pf);
            float ms = 0.0f;
            if (st == MM_OK) st = batch_time(b, reps, e0, e1, &ms);
            if (st == MM_OK && ms < best * 0.99f) {
                best = ms;
                keep = pf;
            }
        }
        for (int c = 0; c < b->n_chains && st == MM_OK; c++)
            if (b->S[c] == S) st = mm_batch_set_chain(b, c, b->team[c], keep);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MM_OK) return st;
    if (moves_per_item) *moves_per_item = b->moves_per_item;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm > 0 ? b->ctas_per_sm : b->max_per_sm;
    if (best_ms) *best_ms = best;
    return MM_OK;
}

}  // extern "C"
