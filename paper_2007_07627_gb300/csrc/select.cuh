// Block-wide exact selection used for the medians of the nu rules.
#pragma once

#include "fricp_internal.cuh"

namespace fricp {

// Exact k-th smallest (0-based) of n non-negative doubles by an 8-bit radix
// select over their IEEE bit patterns (monotone for non-negative values).
static __device__ __noinline__ double block_kth(const double *v, int n, int k) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ int s_k;
    if (threadIdx.x == 0) {
        s_prefix = 0ull;
        s_k = k;
    }
    __syncthreads();
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
        __syncthreads();
        const unsigned long long prefix = s_prefix;
        const unsigned long long mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long key = (unsigned long long)__double_as_longlong(__ldcg(v + i));
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255ull], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned kk = (unsigned)s_k;
            unsigned cum = 0;
            int b = 0;
            for (; b < 255; ++b) {
                if (cum + hist[b] > kk) break;
                cum += hist[b];
            }
            s_k = (int)(kk - cum);
            s_prefix = prefix | ((unsigned long long)b << shift);
        }
        __syncthreads();
    }
    return __longlong_as_double((long long)s_prefix);
}

}  // namespace fricp
