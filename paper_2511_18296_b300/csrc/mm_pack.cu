// Compact 4-byte moves (host-to-device transfer at half the bytes):
// p = (b1 << 16) | code, code < B a swap partner, code = 65535 - t a shift to
// period t (0..T); anything else decodes to the bad move {-1, -1}.
#include "mm_internal.cuh"
#include "mm_move.cuh"

namespace mm {

__global__ void __launch_bounds__(256) k_unpack_moves(const uint32_t *__restrict__ packed, int64_t n, int32_t B,
                                                      int32_t T, int2 *__restrict__ moves) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        moves[i] = unpack_move(__ldg(packed + i), B, T);
    }
}

}  // namespace mm

using namespace mm;

extern "C" mm_status mm_unpack_moves(mm_model *m, const uint32_t *packed, int64_t n, mm_move *moves) {
    if (!m) return set_error(MM_ERR_INVALID_ARG, "NULL model");
    if (n < 0) return set_error(MM_ERR_INVALID_ARG, "negative move count");
    if ((int64_t)m->B + m->T + 1 > 65536)
        return set_error(MM_ERR_INVALID_ARG, "packed moves need B + T + 1 <= 65536 (B = %d, T = %d)", m->B, m->T);
    if (n == 0) return MM_OK;
    if (!packed || !moves) return set_error(MM_ERR_INVALID_ARG, "NULL packed or move pointer");
    if (((uintptr_t)packed & 3u) != 0 || ((uintptr_t)moves & 7u) != 0)
        return set_error(MM_ERR_INVALID_ARG, "packed moves must be 4-byte and moves 8-byte aligned");
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)m->num_sms * 8) blocks = (int64_t)m->num_sms * 8;
    k_unpack_moves<<<(unsigned)blocks, 256, 0, m->stream>>>(packed, n, m->B, m->T, reinterpret_cast<int2 *>(moves));
    return check_launch("k_unpack_moves");
}
