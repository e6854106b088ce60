// Block-wide bitonic sort of 64-bit keys in shared memory (largest first).
#pragma once

#include <cstdint>

namespace mm {

// Descending bitonic sort of s[0..N), N a power of two.
static __device__ __noinline__ void bitonic_desc(uint64_t *s, int N) {
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool desc = ((lo & size) == 0);
                uint64_t a = s[lo], b = s[hi];
                if (desc ? (a < b) : (a > b)) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
        }
    }
    __syncthreads();
}

}  // namespace mm
