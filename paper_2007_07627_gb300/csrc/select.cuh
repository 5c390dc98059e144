// Block-wide exact selection used for the medians of the nu rules.
#pragma once

#include "fricp_internal.cuh"

namespace fricp {

// The two middle order statistics of n non-negative doubles -- the (n-1)/2-th
// and the n/2-th smallest (0-based; equal for odd n) -- found together by an
// 8-bit radix select over their IEEE bit patterns (monotone for non-negative
// values): eight passes over v, each building one histogram per rank of the
// keys that still match that rank's prefix. A warp adds its matching keys per
// bin with one atomic (peers found with __match_any_sync), and warps 0 and 1
// locate their rank's bin with a warp scan. Any blockDim that is a multiple of
// 32 and at least 64 works. The median of v is 0.5 * (*lo + *hi).
static __device__ __noinline__ void block_median_pair(const double *v, int n, double *lo, double *hi) {
    __shared__ unsigned int hist[2][256];
    __shared__ unsigned long long s_prefix[2];
    __shared__ int s_k[2];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_prefix[0] = s_prefix[1] = 0ull;
        s_k[0] = (n - 1) / 2;
        s_k[1] = n / 2;
    }
    __syncthreads();
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 512; b += blockDim.x) (&hist[0][0])[b] = 0u;
        __syncthreads();
        const unsigned long long p0 = s_prefix[0], p1 = s_prefix[1];
        const unsigned long long mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
        for (int base = 0; base < n; base += blockDim.x) {   // every lane runs every round
            const int i = base + threadIdx.x;
            unsigned long long key = ~0ull;
            if (i < n) key = (unsigned long long)__double_as_longlong(__ldcg(v + i));
            const int bin = (int)((key >> shift) & 255ull);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const bool match = i < n && (key & mask) == (r ? p1 : p0);
                const unsigned peers = __match_any_sync(FULL, match ? bin : -1);
                if (match && lane == __ffs(peers) - 1) atomicAdd(&hist[r][bin], (unsigned)__popc(peers));
            }
        }
        __syncthreads();
        if (w < 2) {   // warp r finds the bin holding its rank
            unsigned c[8], s = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = hist[w][8 * lane + q];
                s += c[q];
            }
            unsigned incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const unsigned excl = incl - s;
            const unsigned k = (unsigned)s_k[w];
            const unsigned owner = __ballot_sync(FULL, excl <= k && k < incl);
            if (lane == __ffs(owner) - 1) {
                unsigned cum = excl;
                int q = 0;
                for (; q < 7; ++q) {
                    if (cum + c[q] > k) break;
                    cum += c[q];
                }
                s_k[w] = (int)(k - cum);
                s_prefix[w] |= (unsigned long long)(8 * lane + q) << shift;
            }
        }
        __syncthreads();
    }
    *lo = __longlong_as_double((long long)s_prefix[0]);
    *hi = __longlong_as_double((long long)s_prefix[1]);
}

}  // namespace fricp
