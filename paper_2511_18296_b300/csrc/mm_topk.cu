// Exact, deterministic per-batch top-k of feasible moves.
//
// Each candidate gets a unique 64-bit key: the order-preserving bit pattern of
// its FP32 score (-0 folded into +0) in the high word and the complement of its
// move index in the low word, so larger keys are better and equal scores prefer
// the lower index.  Selection runs in two launches:
//   k_topk_hist    every CTA builds a 4,096-bin shared-memory histogram of the
//                  key's top 12 bits and adds it to a global one; the last CTA to
//                  finish (ticket counter, no waiting) finds the cut-off bin
//                  that holds the k-th best key and clears the histogram.
//   k_topk_collect every CTA appends keys above the cut-off bin to a "sure"
//                  list (< k keys) and keys inside it to a "maybe" list; the
//                  last CTA radix-selects the missing keys from the maybe list
//                  on the remaining 52 bits, sorts the k keys (bitonic, in
//                  shared memory) and writes indices, scores and the count.
// Integer keys make the result independent of thread scheduling.
#include <mutex>

#include "mm_internal.cuh"
#include "mm_sort.cuh"

namespace mm {

enum { kCtlTicket1 = 0, kCtlTakeAll = 1, kCtlCut = 2, kCtlSure = 4, kCtlMaybe = 5, kCtlTicket2 = 6, kCtlWords = 8 };

__device__ __forceinline__ bool make_key(const float *score, const uint8_t *feas, int64_t i, uint64_t &key) {
    if (!feas[i]) return false;
    float f = score[i];
    if (isnan(f)) return false;
    uint32_t u = __float_as_uint(f);
    if ((u << 1) == 0) u = 0;  // -0 -> +0
    uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    key = ((uint64_t)ord << 32) | (uint32_t)(~(uint32_t)i);
    return true;
}

__global__ void __launch_bounds__(256) k_topk_hist(const float *__restrict__ score, const uint8_t *__restrict__ feas,
                                                   int64_t n, int32_t k, uint32_t *__restrict__ hist,
                                                   uint32_t *__restrict__ ctl) {
    __shared__ uint32_t s_h[kHistBins];
    for (int j = threadIdx.x; j < kHistBins; j += blockDim.x) s_h[j] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t key;
        if (make_key(score, feas, i, key)) atomicAdd(&s_h[key >> (64 - kHistBits)], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kHistBins; j += blockDim.x)
        if (s_h[j]) atomicAdd(hist + j, s_h[j]);
    __threadfence();
    __shared__ uint32_t s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ctl + kCtlTicket1, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last CTA: bins scanned from the top; thread t owns the 16 bins
    // [4095 - 16 t - 15, 4095 - 16 t], read as four 16-byte loads.
    static_assert(kHistBins == 16 * 256, "one thread per 16 bins");
    __shared__ uint32_t s_part[256];
    __shared__ uint32_t s_sel[2];  // owner thread, count before it
    const int t = threadIdx.x;
    const int lo_bin = kHistBins - 16 * (t + 1);
    uint32_t h[16];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        uint4 v = __ldcg(reinterpret_cast<const uint4 *>(hist + lo_bin) + q);
        h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
    }
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < 16; j++) local += h[j];
    s_part[t] = local;
    __syncthreads();
    if (t == 0) {
        uint64_t cum = 0, total = 0;
        for (int j = 0; j < 256; j++) total += s_part[j];
        if (total <= (uint64_t)k) {
            ctl[kCtlTakeAll] = 1;
            s_sel[0] = 0xffffffffu;
        } else {
            ctl[kCtlTakeAll] = 0;
            int owner = 255;
            for (int j = 0; j < 256; j++) {
                if (cum + s_part[j] >= (uint64_t)k) { owner = j; break; }
                cum += s_part[j];
            }
            s_sel[0] = (uint32_t)owner;
            s_sel[1] = (uint32_t)cum;
        }
    }
    __syncthreads();
    if (s_sel[0] == (uint32_t)t) {
        uint32_t cum = s_sel[1];
        for (int j = 15; j >= 0; j--) {
            if (cum + h[j] >= (uint32_t)k) {
                ctl[kCtlCut] = (uint32_t)(lo_bin + j);
                break;
            }
            cum += h[j];
        }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) reinterpret_cast<uint4 *>(hist + lo_bin)[q] = make_uint4(0, 0, 0, 0);
    if (t == 0) ctl[kCtlTicket1] = 0;
}

__global__ void __launch_bounds__(256) k_topk_collect(const float *__restrict__ score,
                                                      const uint8_t *__restrict__ feas, int64_t n, int32_t k,
                                                      uint64_t *__restrict__ sure, uint64_t *__restrict__ maybe,
                                                      int64_t cap_maybe, uint32_t *__restrict__ ctl,
                                                      int32_t *__restrict__ idx_out, float *__restrict__ top_out,
                                                      int32_t *__restrict__ count_out) {
    const uint32_t take_all = ctl[kCtlTakeAll];
    const uint32_t cut = ctl[kCtlCut];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t n_round = (n + 31) & ~(int64_t)31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        uint64_t key = 0;
        bool ok = i < n && make_key(score, feas, i, key);
        uint32_t bin = (uint32_t)(key >> (64 - kHistBits));
        bool is_sure = ok && (take_all || bin > cut);
        bool is_maybe = ok && !take_all && bin == cut;
        uint32_t ms = __ballot_sync(0xffffffffu, is_sure);
        uint32_t mm_ = __ballot_sync(0xffffffffu, is_maybe);
        uint32_t base_s = 0, base_m = 0;
        if (lane == 0) {
            if (ms) base_s = atomicAdd(ctl + kCtlSure, __popc(ms));
            if (mm_) base_m = atomicAdd(ctl + kCtlMaybe, __popc(mm_));
        }
        base_s = __shfl_sync(0xffffffffu, base_s, 0);
        base_m = __shfl_sync(0xffffffffu, base_m, 0);
        const uint32_t below = (1u << lane) - 1u;
        if (is_sure) {
            uint32_t pos = base_s + __popc(ms & below);
            if (pos < (uint32_t)kTopkMax) sure[pos] = key;
        }
        if (is_maybe) {
            uint64_t pos = base_m + __popc(mm_ & below);
            if ((int64_t)pos < cap_maybe) maybe[pos] = key;
        }
    }
    __threadfence();
    __shared__ uint32_t s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ctl + kCtlTicket2, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    __shared__ uint64_t s_keys[kTopkMax];
    __shared__ uint32_t s_hist[256];
    __shared__ uint32_t s_n, s_need, s_done;
    __shared__ uint64_t s_prefix, s_mask;
    uint32_t ns = __ldcg(ctl + kCtlSure);
    if (ns > (uint32_t)kTopkMax) ns = kTopkMax;
    uint64_t nm = __ldcg(ctl + kCtlMaybe);
    if ((int64_t)nm > cap_maybe) nm = (uint64_t)cap_maybe;
    for (uint32_t j = threadIdx.x; j < ns; j += blockDim.x) s_keys[j] = __ldcg(sure + j);
    const uint32_t need = take_all ? 0u : (uint32_t)k - ns;
    if (threadIdx.x == 0) {
        s_n = ns;
        s_need = need;
        s_done = 0;
        s_prefix = 0;
        s_mask = 0;
    }
    __syncthreads();
    if (need > 0) {
        if (nm <= need) {
            for (uint32_t j = threadIdx.x; j < (uint32_t)nm; j += blockDim.x) s_keys[ns + j] = __ldcg(maybe + j);
            __syncthreads();
            if (threadIdx.x == 0) s_n = ns + (uint32_t)nm;
        } else {
            // radix select of the `need` largest maybe keys on bits 51..0
            // (digits of 8 bits at shifts 44, 36, ..., 4, then 4 bits at 0)
            int shift = 64 - kHistBits - 8;
            for (; shift > -8; shift -= 8) {
                const int sh = shift < 0 ? 0 : shift;
                for (int j = threadIdx.x; j < 256; j += blockDim.x) s_hist[j] = 0;
                __syncthreads();
                const uint64_t mask = s_mask, prefix = s_prefix;
                for (uint64_t j = threadIdx.x; j < nm; j += blockDim.x) {
                    uint64_t key = __ldcg(maybe + j);
                    if ((key & mask) == prefix) atomicAdd(&s_hist[(key >> sh) & 0xffu], 1u);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t r = s_need, cum = 0;
                    int dgt = 0;
                    for (int b = 255; b >= 0; b--) {
                        if (cum + s_hist[b] >= r) { dgt = b; break; }
                        cum += s_hist[b];
                    }
                    s_need = r - cum;
                    s_prefix = prefix | ((uint64_t)dgt << sh);
                    s_mask = mask | ((0xffull << sh) & ((1ull << (64 - kHistBits)) - 1));
                    s_done = (s_hist[dgt] == s_need) ? 1u : 0u;
                }
                __syncthreads();
                if (s_done) break;
            }
            // keys strictly above the prefix on the selected bits, plus the
            // prefix bin itself (exactly `need` keys in total)
            const uint64_t mask = s_mask, prefix = s_prefix;
            for (uint64_t j = threadIdx.x; j < nm; j += blockDim.x) {
                uint64_t key = __ldcg(maybe + j);
                if ((key & mask) >= prefix) {
                    uint32_t pos = atomicAdd(&s_n, 1u);
                    if (pos < (uint32_t)kTopkMax) s_keys[pos] = key;
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    uint32_t cnt = s_n;
    if (cnt > (uint32_t)k) cnt = (uint32_t)k;
    int N = 1;
    while (N < (int)s_n) N <<= 1;
    for (int j = (int)s_n + threadIdx.x; j < N; j += blockDim.x) s_keys[j] = 0;
    bitonic_desc(s_keys, N);
    for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
        uint32_t id = ~(uint32_t)(s_keys[j] & 0xffffffffull);
        idx_out[j] = (int32_t)id;
        top_out[j] = score[id];
    }
    if (threadIdx.x == 0) {
        *count_out = (int32_t)cnt;
        ctl[kCtlSure] = 0;
        ctl[kCtlMaybe] = 0;
        ctl[kCtlTicket2] = 0;
    }
}

void topk_scratch_free(TopkScratch &scr) {
    cudaFree(scr.hist);
    cudaFree(scr.sure);
    cudaFree(scr.maybe);
    cudaFree(scr.ctl);
    scr = TopkScratch();
}

mm_status topk_scratch_reserve(TopkScratch &scr, int64_t n) {
    if (scr.hist && scr.cap_maybe >= n) return MM_OK;
    int64_t cap = n < 4096 ? 4096 : n;
    if (scr.hist) {
        cudaFree(scr.maybe);
        scr.maybe = nullptr;
        MM_CUDA_TRY(cudaMalloc(&scr.maybe, sizeof(uint64_t) * (size_t)cap), "allocate top-k scratch");
        scr.cap_maybe = cap;
        return MM_OK;
    }
    MM_CUDA_TRY(cudaMalloc(&scr.hist, sizeof(uint32_t) * kHistBins), "allocate top-k scratch");
    MM_CUDA_TRY(cudaMalloc(&scr.sure, sizeof(uint64_t) * kTopkMax), "allocate top-k scratch");
    MM_CUDA_TRY(cudaMalloc(&scr.maybe, sizeof(uint64_t) * (size_t)cap), "allocate top-k scratch");
    MM_CUDA_TRY(cudaMalloc(&scr.ctl, sizeof(uint32_t) * kCtlWords), "allocate top-k scratch");
    MM_CUDA_TRY(cudaMemset(scr.hist, 0, sizeof(uint32_t) * kHistBins), "clear top-k scratch");
    MM_CUDA_TRY(cudaMemset(scr.ctl, 0, sizeof(uint32_t) * kCtlWords), "clear top-k scratch");
    MM_CUDA_TRY(cudaDeviceSynchronize(), "synchronize");
    scr.cap_maybe = cap;
    return MM_OK;
}

mm_status topk_launch(const float *score, const uint8_t *feas, int64_t n, int32_t k, int32_t *idx, float *top,
                      int32_t *count, TopkScratch &scr, int num_sms, cudaStream_t st) {
    if (n == 0) {
        MM_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int32_t), st), "clear count");
        return MM_OK;
    }
    int64_t blocks = (n + 2047) / 2048;
    int64_t cap = (int64_t)num_sms * 2;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_topk_hist<<<(unsigned)blocks, 256, 0, st>>>(score, feas, n, k, scr.hist, scr.ctl);
    mm_status s = check_launch("k_topk_hist");
    if (s != MM_OK) return s;
    k_topk_collect<<<(unsigned)blocks, 256, 0, st>>>(score, feas, n, k, scr.sure, scr.maybe, scr.cap_maybe, scr.ctl,
                                                     idx, top, count);
    return check_launch("k_topk_collect");
}

}  // namespace mm

using namespace mm;

extern "C" mm_status mm_topk(mm_model *m, const float *score, const uint8_t *feas, int64_t n, int32_t k, int32_t *idx,
                             float *top, int32_t *count) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (n < 0 || n > 0x7fffffffLL) return set_error(MM_ERR_INVALID_ARG, "move count out of range");
    if (k < 1 || k > kTopkMax) return set_error(MM_ERR_INVALID_ARG, "k = %d outside 1..%d", k, kTopkMax);
    if (!count || (n > 0 && (!score || !feas || !idx || !top)))
        return set_error(MM_ERR_INVALID_ARG, "NULL pointer");
    if (k <= 32 && n > 0) return topk_small_launch(m, score, feas, n, k, idx, top, count);
    mm_status st = topk_scratch_reserve(m->topk, n);
    if (st != MM_OK) return st;
    return topk_launch(score, feas, n, k, idx, top, count, m->topk, m->num_sms, m->stream);
}

// ---------------------------------------------------------------------------
// Caller-free variant.  Its scratch is one file-scope device array, so a call
// allocates nothing: the array exists on every GPU that loads this library
// until the process exits.  Layout inside the array (byte offsets):
//   [0, 8 MiB)            keys inside the cut-off bin (kNoAllocMaxN x 8 bytes)
//   [8 MiB, +16 KiB)      coarse histogram
//   [+16 KiB, +24 KiB)    keys above the cut-off bin
//   [+24 KiB, +24.25 KiB) counters and tickets
namespace mm {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 20;  // largest batch mm_topk_noalloc accepts
constexpr size_t kNaMaybeOff = 0;
constexpr size_t kNaHistOff = kNaMaybeOff + sizeof(uint64_t) * (size_t)kNoAllocMaxN;
constexpr size_t kNaSureOff = kNaHistOff + sizeof(uint32_t) * kHistBins;
constexpr size_t kNaCtlOff = kNaSureOff + sizeof(uint64_t) * kTopkMax;
constexpr size_t kNaBytes = kNaCtlOff + 256;

static __device__ __align__(256) unsigned char g_topk_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
static std::mutex g_na_mu;
static unsigned char *g_na_base[kNaMaxDevices];  // device address of the array, per device
static int g_na_sms[kNaMaxDevices];

}  // namespace mm

extern "C" mm_status mm_topk_noalloc(const float *score, const uint8_t *feas, int64_t n, int32_t k, int32_t *idx,
                                     float *top, int32_t *count, void *cuda_stream) {
    if (n < 0 || n > kNoAllocMaxN)
        return set_error(MM_ERR_INVALID_ARG, "mm_topk_noalloc: n = %lld is outside 0..%lld (the fixed scratch size)",
                         (long long)n, (long long)kNoAllocMaxN);
    if (k < 1 || k > kTopkMax) return set_error(MM_ERR_INVALID_ARG, "k = %d outside 1..%d", k, kTopkMax);
    if (!count || (n > 0 && (!score || !feas || !idx || !top))) return set_error(MM_ERR_INVALID_ARG, "NULL pointer");
    int dev = 0;
    MM_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kNaMaxDevices) return set_error(MM_ERR_INVALID_ARG, "device %d not supported", dev);
    unsigned char *base;
    int sms;
    {
        // once per device, with that device current: the host-side symbol is not
        // a device address, so ask the runtime for the array's device address
        std::lock_guard<std::mutex> lock(g_na_mu);
        if (!g_na_base[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_topk_noalloc_scratch);
            if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(top-k scratch)");
            int nsm = 0;
            e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return cuda_status(e, "cudaDeviceGetAttribute");
            g_na_sms[dev] = nsm;
            g_na_base[dev] = static_cast<unsigned char *>(p);
        }
        base = g_na_base[dev];
        sms = g_na_sms[dev];
    }
    TopkScratch scr;
    scr.maybe = reinterpret_cast<uint64_t *>(base + kNaMaybeOff);
    scr.hist = reinterpret_cast<uint32_t *>(base + kNaHistOff);
    scr.sure = reinterpret_cast<uint64_t *>(base + kNaSureOff);
    scr.ctl = reinterpret_cast<uint32_t *>(base + kNaCtlOff);
    scr.cap_maybe = kNoAllocMaxN;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: the histogram and the
    // counters must start at zero
    MM_CUDA_TRY(cudaMemsetAsync(scr.hist, 0, kNaCtlOff + 256 - kNaHistOff, st), "clear top-k scratch");
    return topk_launch(score, feas, n, k, idx, top, count, scr, sms, st);
}
