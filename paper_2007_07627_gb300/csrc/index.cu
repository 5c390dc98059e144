// Target index build, source preparation and the target's nu_min statistic.
//
// The exact closest-point query (Sec. 3, Eq. 3) runs over a complete binary
// tree of axis-aligned boxes whose leaves are buckets of kLeaf consecutive
// target points in Morton order. The tree is implicit (node i has children 2i
// and 2i+1), so building it is: bounding box -> 30-bit Morton keys -> radix sort
// -> gather into float4 -> leaf boxes -> one pass per tree level.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fricp_internal.cuh"

namespace fricp {

namespace {

constexpr int kRedBlock = 256;

struct BoxPartial {
    float lo[3], hi[3];
    double sum[3];
    int bad;
};

// Per-block min/max/sum in a fixed order; flags NaN/Inf coordinates and normals
// that are not unit length within 1e-3.
__global__ void k_box_partial(const float *__restrict__ x, const float *__restrict__ nrm, int64_t n,
                              BoxPartial *out, int zero_normals_ok) {
    __shared__ float slo[3][kRedBlock], shi[3][kRedBlock];
    __shared__ double ssum[3][kRedBlock];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double sm[3] = {0.0, 0.0, 0.0};
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        for (int a = 0; a < 3; ++a) {
            const float v = x[3 * i + a];
            if (!isfinite(v)) bad = 1;
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
            sm[a] += (double)v;
        }
        if (nrm != nullptr) {
            const double a0 = nrm[3 * i], a1 = nrm[3 * i + 1], a2 = nrm[3 * i + 2];
            const double l2 = a0 * a0 + a1 * a1 + a2 * a2;
            if (!(fabs(l2 - 1.0) <= 2e-3) && !(zero_normals_ok && l2 == 0.0)) bad = 1;
        }
    }
    __syncthreads();
    if (bad) atomicOr(&sbad, 1);
    for (int a = 0; a < 3; ++a) {
        slo[a][threadIdx.x] = lo[a];
        shi[a][threadIdx.x] = hi[a];
        ssum[a][threadIdx.x] = sm[a];
    }
    __syncthreads();
    for (int s = kRedBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int a = 0; a < 3; ++a) {
                slo[a][threadIdx.x] = fminf(slo[a][threadIdx.x], slo[a][threadIdx.x + s]);
                shi[a][threadIdx.x] = fmaxf(shi[a][threadIdx.x], shi[a][threadIdx.x + s]);
                ssum[a][threadIdx.x] += ssum[a][threadIdx.x + s];
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        BoxPartial r;
        for (int a = 0; a < 3; ++a) {
            r.lo[a] = slo[a][0];
            r.hi[a] = shi[a][0];
            r.sum[a] = ssum[a][0];
        }
        r.bad = sbad;
        out[blockIdx.x] = r;
    }
}

// One block folds the per-block records: thread t takes records t, t+256, ...,
// then a fixed shared-memory tree (deterministic order).
__global__ void k_box_final(const BoxPartial *parts, int nparts, BoxPartial *out) {
    __shared__ float slo[3][kRedBlock], shi[3][kRedBlock];
    __shared__ double ssum[3][kRedBlock];
    __shared__ int sbad[kRedBlock];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double sm[3] = {0.0, 0.0, 0.0};
    int bad = 0;
    for (int b = threadIdx.x; b < nparts; b += kRedBlock) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], parts[b].lo[a]);
            hi[a] = fmaxf(hi[a], parts[b].hi[a]);
            sm[a] += parts[b].sum[a];
        }
        bad |= parts[b].bad;
    }
    for (int a = 0; a < 3; ++a) {
        slo[a][threadIdx.x] = lo[a];
        shi[a][threadIdx.x] = hi[a];
        ssum[a][threadIdx.x] = sm[a];
    }
    sbad[threadIdx.x] = bad;
    __syncthreads();
    for (int s = kRedBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int a = 0; a < 3; ++a) {
                slo[a][threadIdx.x] = fminf(slo[a][threadIdx.x], slo[a][threadIdx.x + s]);
                shi[a][threadIdx.x] = fmaxf(shi[a][threadIdx.x], shi[a][threadIdx.x + s]);
                ssum[a][threadIdx.x] += ssum[a][threadIdx.x + s];
            }
            sbad[threadIdx.x] |= sbad[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        BoxPartial r;
        for (int a = 0; a < 3; ++a) {
            r.lo[a] = slo[a][0];
            r.hi[a] = shi[a][0];
            r.sum[a] = ssum[a][0];
        }
        r.bad = sbad[0];
        *out = r;
    }
}

__device__ __forceinline__ unsigned expand_bits10(unsigned v) {
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__global__ void k_morton(const float *__restrict__ x, int64_t n, float3 lo, float3 inv_ext,
                         unsigned *__restrict__ code, int *__restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float c[3] = {(x[3 * i] - lo.x) * inv_ext.x, (x[3 * i + 1] - lo.y) * inv_ext.y,
                        (x[3 * i + 2] - lo.z) * inv_ext.z};
    unsigned k[3];
    for (int a = 0; a < 3; ++a) k[a] = (unsigned)fminf(fmaxf(c[a] * 1024.0f, 0.0f), 1023.0f);
    code[i] = (expand_bits10(k[0]) << 2) | (expand_bits10(k[1]) << 1) | expand_bits10(k[2]);
    idx[i] = (int)i;
}

__global__ void k_gather(const float *__restrict__ x, const float *__restrict__ nrm, const int *__restrict__ order,
                         int64_t n, float4 *__restrict__ pts, float4 *__restrict__ nout) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int o = order[i];
    pts[i] = make_float4(x[3 * (int64_t)o], x[3 * (int64_t)o + 1], x[3 * (int64_t)o + 2], __int_as_float(o));
    if (nrm != nullptr && nout != nullptr)
        nout[i] = make_float4(nrm[3 * (int64_t)o], nrm[3 * (int64_t)o + 1], nrm[3 * (int64_t)o + 2], 0.0f);
}

__global__ void k_leaf_boxes(const float4 *__restrict__ pts, int64_t n, int L, float4 *__restrict__ nodes) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
    const int64_t beg = (int64_t)l * kLeaf;
    const int64_t end = beg + kLeaf < n ? beg + kLeaf : n;
    for (int64_t j = beg; j < end; ++j) {
        const float4 p = pts[j];
        lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
        hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
    }
    const int node = L + l;
    nodes[2 * node] = lo;
    nodes[2 * node + 1] = hi;
}

// Oriented box of every bucket (obb_fit in obb.cuh), the bound obb_d2 tests.
// Empty buckets get a zero box: their axis-aligned box (inverted) already fails
// every test.
__global__ void k_leaf_obb(const float4 *__restrict__ pts, int64_t n, int L, float4 *__restrict__ obb) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    float4 *o = obb + 4 * (int64_t)l;
    const int64_t beg = (int64_t)l * kLeaf;
    const int64_t end = beg + kLeaf < n ? beg + kLeaf : n;
    if (beg >= end) {
        for (int k = 0; k < 4; ++k) o[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        return;
    }
    float4 box[4];
    obb_fit(pts + beg, (int)(end - beg), box);
    for (int k = 0; k < 4; ++k) o[k] = box[k];
}

__global__ void k_level_boxes(float4 *__restrict__ nodes, int first, int count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int i = first + k;
    const float4 a0 = nodes[4 * i], a1 = nodes[4 * i + 1], b0 = nodes[4 * i + 2], b1 = nodes[4 * i + 3];
    nodes[2 * i] = make_float4(fminf(a0.x, b0.x), fminf(a0.y, b0.y), fminf(a0.z, b0.z), 0.0f);
    nodes[2 * i + 1] = make_float4(fmaxf(a1.x, b1.x), fmaxf(a1.y, b1.y), fmaxf(a1.z, b1.z), 0.0f);
}

// Six nearest target points of every target point, the point itself excluded
// (duplicates at distance zero count), ordered by (exact FP64 squared distance,
// original index). Per point: the median of the six distances (Sec. 4.3) and,
// with normals, the median of the six distances to the point's tangent plane
// (Sec. 5); the median of six is the mean of the 3rd and 4th smallest.
//
// One warp per query point, the traversal of warp_nn: the query's own bucket
// is scanned first, then the siblings of its path to the root and what they
// open, two tree levels per round; lanes test boxes and bucket points in
// parallel. Pruning is in float: a box or candidate is skipped only when its
// float squared distance, shrunk by kShrink (far more than the float rounding
// of either), exceeds the current sixth-best FP64 distance rounded up to float.
// Every point that can enter the six gets its exact FP64 distance, and the six
// (kept identical in every lane) are merged one at a time in a fixed order, so
// the selection and the medians are exact.
struct Best6 {
    double d[6];
    int o[6], j[6];
    float bound;   // d[5] rounded up to float
};

// Insert (d, o, j) into the six kept in (d, o) order, if it belongs there. Fully
// unrolled with constant indices, so the six stay in registers: slot s takes
// the old entry s - 1 while that one orders after the newcomer, the newcomer at
// the first slot where it does not, and slot 0 if it orders before all.
__device__ __forceinline__ void best6_insert(Best6 &b, double d, int o, int j) {
    if (!(d < b.d[5] || (d == b.d[5] && o < b.o[5]))) return;
    bool done = false;
#pragma unroll
    for (int s = 5; s >= 1; --s) {
        const bool after = !done && (b.d[s - 1] > d || (b.d[s - 1] == d && b.o[s - 1] > o));
        const bool put = !done && !after;
        b.d[s] = after ? b.d[s - 1] : (put ? d : b.d[s]);
        b.o[s] = after ? b.o[s - 1] : (put ? o : b.o[s]);
        b.j[s] = after ? b.j[s - 1] : (put ? j : b.j[s]);
        done = done || put;
    }
    if (!done) {
        b.d[0] = d;
        b.o[0] = o;
        b.j[0] = j;
    }
    b.bound = __double2float_ru(b.d[5]);
}

// Offers bucket na's points (lanes 0-15) and, if `two`, bucket nb's (lanes
// 16-31) to the six; the point i itself is skipped.
__device__ __forceinline__ void knn6_scan(const Index &ix, int i, const float xq[3], Best6 &b, int na, int nb,
                                          bool two) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    bool cand = false;
    double d = 0.0;
    int o = 0, j = -1;
    if (lane < 16 || two) {
        j = ((lane < 16 ? na : nb) - ix.L) * kLeaf + (lane & 15);
        if (j < ix.n && j != i) {
            const float4 q = __ldg(ix.pts + j);
            const float fx = q.x - xq[0], fy = q.y - xq[1], fz = q.z - xq[2];
            if (fmaf(fz, fz, fmaf(fy, fy, fx * fx)) * kShrink <= b.bound) {
                const double a0 = (double)q.x - (double)xq[0], a1 = (double)q.y - (double)xq[1],
                             a2 = (double)q.z - (double)xq[2];
                d = a0 * a0 + a1 * a1 + a2 * a2;
                o = __float_as_int(q.w);
                cand = true;
            }
        }
    }
    unsigned cm = __ballot_sync(FULL, cand);
    while (cm) {   // merge in lane order: every lane applies the same insertions
        const int src = __ffs(cm) - 1;
        cm &= cm - 1u;
        const double dv = __shfl_sync(FULL, d, src);
        const int ov = __shfl_sync(FULL, o, src), jv = __shfl_sync(FULL, j, src);
        best6_insert(b, dv, ov, jv);
    }
}

// Returns false if the stack would overflow.
__device__ bool warp_knn6(const Index &ix, int i, const float xq[3], Best6 &b, int *stk) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    for (int s = 0; s < 6; ++s) {
        b.d[s] = INFINITY;
        b.o[s] = 0x7fffffff;
        b.j[s] = -1;
    }
    b.bound = INFINITY;
    int depth = 0;
    while ((1 << depth) < ix.L) ++depth;
    // the query's own bucket and its sibling bucket first: a tight bound early
    const int start = ix.L + i / kLeaf;
    knn6_scan(ix, i, xq, b, start, start ^ 1, depth > 0);   // a one-bucket tree has no sibling
    int sp;
    {
        int c = 0;
        bool pass = false;
        if (lane < depth - 1) {   // the sibling of the path node at level lane + 1 (the bucket level is done)
            c = (start >> (depth - 1 - lane)) ^ 1;
            pass = box_d2(__ldg(ix.nodes + 2 * c), __ldg(ix.nodes + 2 * c + 1), xq, zero) * kShrink <= b.bound;
        }
        const unsigned m = __ballot_sync(FULL, pass);
        if (pass) stk[__popc(m & below)] = c;
        sp = __popc(m);
    }
    __syncwarp();
    const int leaf_parent_level = depth - 1;
    while (sp > 0) {
        const int k = min(32, sp);
        const int node = (lane < k) ? stk[sp - 1 - lane] : 0;
        sp -= k;
        __syncwarp();
        int c[4] = {0, 0, 0, 0};
        bool ok[4] = {false, false, false, false};
        bool leaf_ok = false;
        if (node != 0) {
            if (node < ix.L) {
                const int level = 31 - __clz(node);
                if (level < leaf_parent_level) {
                    const float4 *bx = ix.nodes + 8 * node;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        c[g] = 4 * node + g;
                        ok[g] = box_d2(__ldg(bx + 2 * g), __ldg(bx + 2 * g + 1), xq, zero) * kShrink <= b.bound;
                    }
                } else {
                    const float4 *bx = ix.nodes + 4 * node;
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        c[g] = 2 * node + g;
                        ok[g] = box_d2(__ldg(bx + 2 * g), __ldg(bx + 2 * g + 1), xq, zero) * kShrink <= b.bound;
                    }
                }
            } else {
                leaf_ok = box_d2(__ldg(ix.nodes + 2 * node), __ldg(ix.nodes + 2 * node + 1), xq, zero) * kShrink
                              <= b.bound &&
                          (ix.obb == nullptr ||
                           obb_d2(ix.obb + 4 * (node - ix.L), xq, zero) * kObbShrink <= b.bound);
            }
        }
        int base = sp;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const unsigned mg = __ballot_sync(FULL, ok[g]);
            if (base + __popc(mg) > kWarpStack) return false;
            if (ok[g]) stk[base + __popc(mg & below)] = c[g];
            base += __popc(mg);
        }
        sp = base;
        unsigned lm = __ballot_sync(FULL, leaf_ok);
        while (lm) {   // two buckets per pass: lanes 0-15 and 16-31
            const int la = __ffs(lm) - 1;
            lm &= lm - 1u;
            int lb = la;
            bool two = false;
            if (lm) {
                lb = __ffs(lm) - 1;
                lm &= lm - 1u;
                two = true;
            }
            const int na = __shfl_sync(FULL, node, la), nb = __shfl_sync(FULL, node, lb);
            knn6_scan(ix, i, xq, b, na, nb, two);
        }
        __syncwarp();
    }
    return true;
}

constexpr int kKnnBlock = 128;

// Per-point statistics of point i from its six nearest (Sec. 4.3, Sec. 5): the
// median of the six distances and, with normals, of the six distances to the
// point's tangent plane (the median of six: the mean of the 3rd and 4th).
__device__ void write_knn6_stats(const Index &ix, int i, const float xq[3], const Best6 &b, double *stat_d,
                                 double *stat_h) {
    const double x0 = xq[0], x1 = xq[1], x2 = xq[2];
    stat_d[i] = 0.5 * (sqrt(b.d[2]) + sqrt(b.d[3]));
    if (stat_h != nullptr) {
        const float4 ni = ix.nrm[i];
        double h[6];
        for (int s = 0; s < 6; ++s) {
            if (b.j[s] < 0) {
                h[s] = INFINITY;
                continue;
            }
            const float4 q = ix.pts[b.j[s]];
            h[s] = fabs(((double)q.x - x0) * ni.x + ((double)q.y - x1) * ni.y + ((double)q.z - x2) * ni.z);
        }
        for (int a = 1; a < 6; ++a) {   // insertion sort of six values
            const double v = h[a];
            int c = a - 1;
            while (c >= 0 && h[c] > v) {
                h[c + 1] = h[c];
                --c;
            }
            h[c + 1] = v;
        }
        stat_h[i] = 0.5 * (h[2] + h[3]);
    }
}

__global__ void __launch_bounds__(kKnnBlock) k_knn6_stats(Index ix, double *__restrict__ stat_d,
                                                          double *__restrict__ stat_h, int *__restrict__ overflow) {
    __shared__ int s_stk[kKnnBlock / 32][kWarpStack];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int wpb = kKnnBlock / 32;
    for (int i = blockIdx.x * wpb + w; i < ix.n; i += gridDim.x * wpb) {
        const float4 qi = __ldg(ix.pts + i);
        const float xq[3] = {qi.x, qi.y, qi.z};
        Best6 b;
        if (!warp_knn6(ix, i, xq, b, s_stk[w])) {
            if (lane == 0) *overflow = 1;
            continue;
        }
        if (lane == 0) write_knn6_stats(ix, i, xq, b, stat_d, stat_h);
    }
}

// Six-neighbour statistics by tiles: a warp takes the 32 Morton-consecutive
// target points of buckets 2g and 2g + 1, one per lane, each lane keeping its
// own six nearest (Best6, the same (FP64 distance, index) order and float
// pre-test as warp_knn6).
//   1. Each lane offers the tile's other 31 points to its six: its sixth
//      distance is then an upper bound of its true sixth distance, and R, the
//      largest over the lanes (rounded up to float), bounds them all.
//   2. Every point within sqrt(R) of some lane's point lies within sqrt(R) of
//      the two buckets' common box (the tree node above them), so the buckets
//      whose box is within that distance of that box (walk from the node's path
//      siblings, box-to-box distance, kShrink slack) hold every candidate.
//   3. Each lane offers the points of those buckets to its six, pruning with
//      its own sixth distance.
// The six selected are therefore the exact six of warp_knn6. A tile whose
// bucket list does not fit (a scattered tile, or fewer than seven points in
// it) is searched point by point with warp_knn6 instead.
constexpr int kKnnCand = 192;   // candidate buckets per tile

__device__ __forceinline__ float box_box_d2(float4 alo, float4 ahi, float4 blo, float4 bhi) {
    const float gx = fmaxf(fmaxf(alo.x - bhi.x, blo.x - ahi.x), 0.0f);
    const float gy = fmaxf(fmaxf(alo.y - bhi.y, blo.y - ahi.y), 0.0f);
    const float gz = fmaxf(fmaxf(alo.z - bhi.z, blo.z - ahi.z), 0.0f);
    return fmaf(gz, gz, fmaf(gy, gy, gx * gx));
}

__device__ __forceinline__ void knn6_offer_own(Best6 &b, float4 q, const float xq[3], int j) {
    const float fx = q.x - xq[0], fy = q.y - xq[1], fz = q.z - xq[2];
    if (fmaf(fz, fz, fmaf(fy, fy, fx * fx)) * kShrink <= b.bound) {
        const double a0 = (double)q.x - (double)xq[0], a1 = (double)q.y - (double)xq[1],
                     a2 = (double)q.z - (double)xq[2];
        best6_insert(b, a0 * a0 + a1 * a1 + a2 * a2, __float_as_int(q.w), j);
    }
}

// Returns false when the candidate list or the walk's stack would overflow.
__device__ bool tile_knn6(const Index &ix, int g, int i, bool live, const float xq[3], Best6 &b, int *stk,
                          int *cand) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    for (int s = 0; s < 6; ++s) {
        b.d[s] = INFINITY;
        b.o[s] = 0x7fffffff;
        b.j[s] = -1;
    }
    b.bound = INFINITY;
    const int i0 = 32 * g;
    const float4 mine = live ? __ldg(ix.pts + i) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int k = 1; k < 32; ++k) {   // 1. the tile's own points, nearest in Morton order first
        const int off = (k & 1) ? (k + 1) >> 1 : -(k >> 1);   // +1, -1, +2, -2, ..., -15, +16
        const int t = (lane + off) & 31;
        float4 q;
        q.x = __shfl_sync(FULL, mine.x, t);
        q.y = __shfl_sync(FULL, mine.y, t);
        q.z = __shfl_sync(FULL, mine.z, t);
        q.w = __shfl_sync(FULL, mine.w, t);
        if (live && i0 + t < ix.n) knn6_offer_own(b, q, xq, i0 + t);
    }
    float R = live ? b.bound : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) R = fmaxf(R, __shfl_xor_sync(FULL, R, o));
    if (!(R < INFINITY)) return false;
    // 2. buckets within sqrt(R) of the tile's box (node P above buckets 2g, 2g + 1)
    int depth = 0;
    while ((1 << depth) < ix.L) ++depth;
    const int P = (ix.L >> 1) + g;
    const float4 glo = __ldg(ix.nodes + 2 * P), ghi = __ldg(ix.nodes + 2 * P + 1);
    int sp = 0, nc = 0;
    {
        int c = 0;
        bool pass = false;
        if (lane < depth - 1) {   // siblings of P's path, from the root's children down
            c = (P >> (depth - 2 - lane)) ^ 1;
            pass = box_box_d2(__ldg(ix.nodes + 2 * c), __ldg(ix.nodes + 2 * c + 1), glo, ghi) * kShrink <= R;
        }
        const unsigned m = __ballot_sync(FULL, pass);
        if (pass) stk[__popc(m & below)] = c;
        sp = __popc(m);
    }
    __syncwarp();
    while (sp > 0) {
        const int k = min(32, sp);
        const int node = (lane < k) ? stk[sp - 1 - lane] : 0;
        sp -= k;
        __syncwarp();
        int c[4] = {0, 0, 0, 0};
        bool ok[4] = {false, false, false, false};
        bool leaf = false;
        if (node != 0) {
            if (node < ix.L) {
                const int level = 31 - __clz(node);
                if (level < depth - 1) {
                    const float4 *bx = ix.nodes + 8 * node;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        c[q] = 4 * node + q;
                        ok[q] = box_box_d2(__ldg(bx + 2 * q), __ldg(bx + 2 * q + 1), glo, ghi) * kShrink <= R;
                    }
                } else {
                    const float4 *bx = ix.nodes + 4 * node;
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        c[q] = 2 * node + q;
                        ok[q] = box_box_d2(__ldg(bx + 2 * q), __ldg(bx + 2 * q + 1), glo, ghi) * kShrink <= R;
                    }
                }
            } else {
                leaf = true;   // tested when it was pushed
            }
        }
        const unsigned lm = __ballot_sync(FULL, leaf);
        if (nc + __popc(lm) > kKnnCand) return false;
        if (leaf) cand[nc + __popc(lm & below)] = node;
        nc += __popc(lm);
        int base = sp;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned mq = __ballot_sync(FULL, ok[q]);
            if (base + __popc(mq) > kWarpStack - kKnnCand) return false;
            if (ok[q]) stk[base + __popc(mq & below)] = c[q];
            base += __popc(mq);
        }
        sp = base;
        __syncwarp();
    }
    // 3. every lane offers the candidates' points to its own six, bucket by
    //    bucket; a lane whose own bound the bucket's boxes exceed skips it, and
    //    the warp skips a bucket no lane needs
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < nc; ++k) {
        const int c = cand[k];
        bool need = false;
        if (live)
            need = box_d2(__ldg(ix.nodes + 2 * c), __ldg(ix.nodes + 2 * c + 1), xq, zero) * kShrink <= b.bound &&
                   (ix.obb == nullptr || obb_d2(ix.obb + 4 * (c - ix.L), xq, zero) * kObbShrink <= b.bound);
        if (!__any_sync(FULL, need)) continue;
        const int beg = (c - ix.L) * kLeaf;
        const int end = min(beg + kLeaf, ix.n);
        if (need)
            for (int j = beg; j < end; ++j) knn6_offer_own(b, __ldg(ix.pts + j), xq, j);
    }
    __syncwarp();
    return true;
}

__global__ void __launch_bounds__(kKnnBlock) k_knn6_tile(Index ix, double *__restrict__ stat_d,
                                                         double *__restrict__ stat_h, int *__restrict__ overflow) {
    __shared__ int s_stk[kKnnBlock / 32][kWarpStack];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int wpb = kKnnBlock / 32;
    const int ngroups = (ix.n + 31) / 32;
    int *stk = s_stk[w];
    int *cand = s_stk[w] + (kWarpStack - kKnnCand);
    for (int g = blockIdx.x * wpb + w; g < ngroups; g += gridDim.x * wpb) {
        const int i = 32 * g + lane;
        const bool live = i < ix.n;
        float xq[3] = {0.0f, 0.0f, 0.0f};
        if (live) {
            const float4 qi = __ldg(ix.pts + i);
            xq[0] = qi.x;
            xq[1] = qi.y;
            xq[2] = qi.z;
        }
        Best6 b;
        if (tile_knn6(ix, g, i, live, xq, b, stk, cand)) {
            if (live) write_knn6_stats(ix, i, xq, b, stat_d, stat_h);
            continue;
        }
        __syncwarp();
        for (int t = 0; t < 32 && 32 * g + t < ix.n; ++t) {   // point by point
            const int it = 32 * g + t;
            const float4 qt = __ldg(ix.pts + it);
            const float xt[3] = {qt.x, qt.y, qt.z};
            Best6 bt;
            if (!warp_knn6(ix, it, xt, bt, stk)) {
                if (lane == 0) *overflow = 1;
                continue;
            }
            if (lane == 0) write_knn6_stats(ix, it, xt, bt, stat_d, stat_h);
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Normal estimate (Sec. 6: where the surface is unknown the paper estimates
// normals from the 30 nearest neighbours): the neighbourhood of q_i is its k
// nearest points, q_i included, ordered by (exact FP64 squared distance,
// original index); the normal is the eigenvector of the smallest eigenvalue of
// the neighbourhood's covariance about its centroid, turned towards a viewpoint.
//
// k_knn_cov: one warp per point, the traversal of warp_knn6. The warp keeps the
// sorted k nearest one entry per lane (lane s holds the s-th nearest), inserts a
// candidate with one ballot and one shift, and prunes in float against the k-th
// distance rounded up. Candidate distances are FP64 without fused
// multiply-adds, so the order is that of a plain evaluation of
// (dx^2 + dy^2) + dz^2. Writes the 6 covariance entries per point.
// ---------------------------------------------------------------------------
constexpr int kMaxNormalK = 32;

__device__ __forceinline__ double exact_d2(float4 q, const float xq[3]) {
    const double a0 = (double)q.x - (double)xq[0], a1 = (double)q.y - (double)xq[1], a2 = (double)q.z - (double)xq[2];
    return __dadd_rn(__dadd_rn(__dmul_rn(a0, a0), __dmul_rn(a1, a1)), __dmul_rn(a2, a2));
}

struct TopK {
    double d;   // lane s: the s-th smallest squared distance so far
    int o, j;   // its original index and bucket-order position
    float bound;
};

__device__ __forceinline__ void topk_scan(const Index &ix, const float xq[3], TopK &t, int K, int na, int nb,
                                          bool two) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    bool cand = false;
    double d = 0.0;
    int o = 0, j = -1;
    if (lane < 16 || two) {
        j = ((lane < 16 ? na : nb) - ix.L) * kLeaf + (lane & 15);
        if (j < ix.n) {
            const float4 q = __ldg(ix.pts + j);
            const float fx = q.x - xq[0], fy = q.y - xq[1], fz = q.z - xq[2];
            if (fmaf(fz, fz, fmaf(fy, fy, fx * fx)) * kShrink <= t.bound) {
                d = exact_d2(q, xq);
                o = __float_as_int(q.w);
                cand = true;
            }
        }
    }
    unsigned cm = __ballot_sync(FULL, cand);
    while (cm) {   // insert in lane order
        const int src = __ffs(cm) - 1;
        cm &= cm - 1u;
        const double dv = __shfl_sync(FULL, d, src);
        const int ov = __shfl_sync(FULL, o, src), jv = __shfl_sync(FULL, j, src);
        const bool greater = lane < K && (t.d > dv || (t.d == dv && t.o > ov));
        const unsigned gm = __ballot_sync(FULL, greater);
        if (gm == 0u) continue;   // not among the K nearest
        const int pos = __ffs(gm) - 1;
        const double ud = __shfl_up_sync(FULL, t.d, 1);
        const int uo = __shfl_up_sync(FULL, t.o, 1), uj = __shfl_up_sync(FULL, t.j, 1);
        if (lane == pos) {
            t.d = dv;
            t.o = ov;
            t.j = jv;
        } else if (lane > pos && lane < K) {
            t.d = ud;
            t.o = uo;
            t.j = uj;
        }
        t.bound = __double2float_ru(__shfl_sync(FULL, t.d, K - 1));
    }
}

// Returns false if the stack would overflow.
__device__ bool warp_knn_k(const Index &ix, int i, const float xq[3], int K, TopK &t, int *stk) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    t.d = INFINITY;
    t.o = 0x7fffffff;
    t.j = -1;
    t.bound = INFINITY;
    int depth = 0;
    while ((1 << depth) < ix.L) ++depth;
    const int start = ix.L + i / kLeaf;
    topk_scan(ix, xq, t, K, start, start ^ 1, depth > 0);   // the point's bucket and its sibling first
    int sp;
    {
        int c = 0;
        bool pass = false;
        if (lane < depth - 1) {
            c = (start >> (depth - 1 - lane)) ^ 1;
            pass = box_d2(__ldg(ix.nodes + 2 * c), __ldg(ix.nodes + 2 * c + 1), xq, zero) * kShrink <= t.bound;
        }
        const unsigned m = __ballot_sync(FULL, pass);
        if (pass) stk[__popc(m & below)] = c;
        sp = __popc(m);
    }
    __syncwarp();
    const int leaf_parent_level = depth - 1;
    while (sp > 0) {
        const int k = min(32, sp);
        const int node = (lane < k) ? stk[sp - 1 - lane] : 0;
        sp -= k;
        __syncwarp();
        int c[4] = {0, 0, 0, 0};
        bool ok[4] = {false, false, false, false};
        bool leaf_ok = false;
        if (node != 0) {
            if (node < ix.L) {
                const int level = 31 - __clz(node);
                if (level < leaf_parent_level) {
                    const float4 *bx = ix.nodes + 8 * node;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        c[g] = 4 * node + g;
                        ok[g] = box_d2(__ldg(bx + 2 * g), __ldg(bx + 2 * g + 1), xq, zero) * kShrink <= t.bound;
                    }
                } else {
                    const float4 *bx = ix.nodes + 4 * node;
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        c[g] = 2 * node + g;
                        ok[g] = box_d2(__ldg(bx + 2 * g), __ldg(bx + 2 * g + 1), xq, zero) * kShrink <= t.bound;
                    }
                }
            } else {
                leaf_ok = box_d2(__ldg(ix.nodes + 2 * node), __ldg(ix.nodes + 2 * node + 1), xq, zero) * kShrink
                              <= t.bound &&
                          (ix.obb == nullptr ||
                           obb_d2(ix.obb + 4 * (node - ix.L), xq, zero) * kObbShrink <= t.bound);
            }
        }
        int base = sp;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const unsigned mg = __ballot_sync(FULL, ok[g]);
            if (base + __popc(mg) > kWarpStack) return false;
            if (ok[g]) stk[base + __popc(mg & below)] = c[g];
            base += __popc(mg);
        }
        sp = base;
        unsigned lm = __ballot_sync(FULL, leaf_ok);
        while (lm) {   // two buckets per pass: lanes 0-15 and 16-31
            const int la = __ffs(lm) - 1;
            lm &= lm - 1u;
            int lb = la;
            bool two = false;
            if (lm) {
                lb = __ffs(lm) - 1;
                lm &= lm - 1u;
                two = true;
            }
            const int na = __shfl_sync(FULL, node, la), nb = __shfl_sync(FULL, node, lb);
            topk_scan(ix, xq, t, K, na, nb, two);
        }
        __syncwarp();
    }
    return true;
}

__global__ void __launch_bounds__(kKnnBlock) k_knn_cov(Index ix, int K, double *__restrict__ cov,
                                                       int *__restrict__ overflow) {
    __shared__ int s_stk[kKnnBlock / 32][kWarpStack];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int wpb = kKnnBlock / 32;
    for (int i = blockIdx.x * wpb + w; i < ix.n; i += gridDim.x * wpb) {
        const float4 qi = __ldg(ix.pts + i);
        const float xq[3] = {qi.x, qi.y, qi.z};
        TopK t;
        if (!warp_knn_k(ix, i, xq, K, t, s_stk[w])) {
            if (lane == 0) *overflow = 1;
            continue;
        }
        // centroid and covariance of the K neighbours (lanes 0..K-1), FP64 warp sums
        double p[3] = {0.0, 0.0, 0.0};
        if (lane < K) {
            const float4 q = __ldg(ix.pts + t.j);
            p[0] = q.x;
            p[1] = q.y;
            p[2] = q.z;
        }
        double c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = p[a];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            c[a] = v / (double)K;
        }
        double e[6] = {0, 0, 0, 0, 0, 0};
        if (lane < K) {
            const double x = p[0] - c[0], y = p[1] - c[1], z = p[2] - c[2];
            e[0] = x * x;
            e[1] = x * y;
            e[2] = x * z;
            e[3] = y * y;
            e[4] = y * z;
            e[5] = z * z;
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e[a] += __shfl_xor_sync(0xffffffffu, e[a], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < 6; ++a) cov[6 * (size_t)i + a] = e[a] / (double)K;
        }
    }
}

// Eigenvector of the smallest eigenvalue of each 3x3 covariance (cyclic Jacobi
// in FP64), turned so that n . (viewpoint - q) >= 0, written at the point's
// original index.
__global__ void k_normal_from_cov(Index ix, const double *__restrict__ cov, double v0, double v1, double v2,
                                  float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ix.n) return;
    double a[3][3], V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    const double *e = cov + 6 * (size_t)i;
    a[0][0] = e[0];
    a[0][1] = a[1][0] = e[1];
    a[0][2] = a[2][0] = e[2];
    a[1][1] = e[3];
    a[1][2] = a[2][1] = e[4];
    a[2][2] = e[5];
    const int P[3] = {0, 0, 1}, Qi[3] = {1, 2, 2};
    for (int sweep = 0; sweep < 32; ++sweep) {
        const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        const double diag = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
        if (!(off > 1e-18 * diag)) break;
        for (int r = 0; r < 3; ++r) {
            const int pp = P[r], qq = Qi[r];
            if (a[pp][qq] == 0.0) continue;
            const double th = (a[qq][qq] - a[pp][pp]) / (2.0 * a[pp][qq]);
            const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double cs = 1.0 / sqrt(tt * tt + 1.0), sn = tt * cs;
            for (int k = 0; k < 3; ++k) {   // a <- J^T a J
                const double akp = a[k][pp], akq = a[k][qq];
                a[k][pp] = cs * akp - sn * akq;
                a[k][qq] = sn * akp + cs * akq;
            }
            for (int k = 0; k < 3; ++k) {
                const double apk = a[pp][k], aqk = a[qq][k];
                a[pp][k] = cs * apk - sn * aqk;
                a[qq][k] = sn * apk + cs * aqk;
            }
            for (int k = 0; k < 3; ++k) {   // V <- V J
                const double vkp = V[k][pp], vkq = V[k][qq];
                V[k][pp] = cs * vkp - sn * vkq;
                V[k][qq] = sn * vkp + cs * vkq;
            }
        }
    }
    int m = 0;
    if (a[1][1] < a[m][m]) m = 1;
    if (a[2][2] < a[m][m]) m = 2;
    double n[3] = {V[0][m], V[1][m], V[2][m]};
    const double inv = 1.0 / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const float4 q = __ldg(ix.pts + i);
    const double side = n[0] * (v0 - (double)q.x) + n[1] * (v1 - (double)q.y) + n[2] * (v2 - (double)q.z);
    const double sg = side < 0.0 ? -inv : inv;
    const int o = __float_as_int(q.w);
    out[3 * (size_t)o] = (float)(n[0] * sg);
    out[3 * (size_t)o + 1] = (float)(n[1] * sg);
    out[3 * (size_t)o + 2] = (float)(n[2] * sg);
}

// Grid-wide form of block_median_pair for large n (the nu_min medians of a
// whole target): the same eight 8-bit radix passes over the IEEE bit patterns,
// but each pass's two histograms are built by every block (shared-memory
// histograms folded into MedianState::hist with one atomic per bin and block)
// and one block then locates each rank's bin. Counts do not depend on the
// order of the atomics, so the result is the one block_median_pair gives.
// Launch order: k_median_init, then for shift = 56, 48, ..., 0 one
// k_median_hist and one k_median_pick (64 threads); the last pick writes
// 0.5 * (lo + hi) to *out.
struct MedianState {
    unsigned long long prefix[2];
    int k[2];
    unsigned int hist[2][256];
};

__global__ void k_median_init(MedianState *st, int n) {
    for (int b = threadIdx.x; b < 512; b += blockDim.x) (&st->hist[0][0])[b] = 0u;
    if (threadIdx.x == 0) {
        st->prefix[0] = st->prefix[1] = 0ull;
        st->k[0] = (n - 1) / 2;
        st->k[1] = n / 2;
    }
}

__global__ void k_median_hist(const double *v, int n, MedianState *st, int shift) {
    __shared__ unsigned int hist[2][256];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < 512; b += blockDim.x) (&hist[0][0])[b] = 0u;
    __syncthreads();
    const unsigned long long p0 = st->prefix[0], p1 = st->prefix[1];
    const unsigned long long mask = (shift == 56) ? 0ull : (~0ull << (shift + 8));
    // every lane runs every round (the peer match is warp-wide)
    for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
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
    for (int b = threadIdx.x; b < 512; b += blockDim.x) {
        const unsigned c = (&hist[0][0])[b];
        if (c) atomicAdd(&st->hist[0][0] + b, c);
    }
}

__global__ void __launch_bounds__(64) k_median_pick(MedianState *st, int shift, double *out) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w < 2) {   // warp r finds the bin holding its rank (as block_median_pair)
        unsigned c[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = st->hist[w][8 * lane + q];
            sum += c[q];
        }
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned excl = incl - sum;
        const unsigned k = (unsigned)st->k[w];
        const unsigned owner = __ballot_sync(FULL, excl <= k && k < incl);
        if (lane == __ffs(owner) - 1) {
            unsigned cum = excl;
            int q = 0;
            for (; q < 7; ++q) {
                if (cum + c[q] > k) break;
                cum += c[q];
            }
            st->k[w] = (int)(k - cum);
            st->prefix[w] |= (unsigned long long)(8 * lane + q) << shift;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 512; b += blockDim.x) (&st->hist[0][0])[b] = 0u;   // for the next pass
    if (shift == 0 && threadIdx.x == 0)
        *out = 0.5 * (__longlong_as_double((long long)st->prefix[0]) + __longlong_as_double((long long)st->prefix[1]));
}

struct BoxResult {
    float lo[3], hi[3];
    double sum[3];
    int bad;
};

cudaError_t reduce_box(const float *x, const float *nrm, int64_t n, cudaStream_t s, BoxResult *res,
                       int zero_normals_ok = 0) {
    int nb = (int)std::min<int64_t>((n + kRedBlock - 1) / kRedBlock, 1024);
    if (nb < 1) nb = 1;
    BoxPartial *parts = nullptr;
    cudaError_t e = cudaMallocAsync(&parts, sizeof(BoxPartial) * (nb + 1), s);
    if (e != cudaSuccess) return e;
    k_box_partial<<<nb, kRedBlock, 0, s>>>(x, nrm, n, parts, zero_normals_ok);
    k_box_final<<<1, kRedBlock, 0, s>>>(parts, nb, parts + nb);
    counters().launches += 2;
    BoxPartial h;
    e = cudaMemcpyAsync(&h, parts + nb, sizeof(BoxPartial), cudaMemcpyDeviceToHost, s);
    counters().d2h += sizeof(BoxPartial);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(parts, s);
    if (e != cudaSuccess) return e;
    for (int a = 0; a < 3; ++a) {
        res->lo[a] = h.lo[a];
        res->hi[a] = h.hi[a];
        res->sum[a] = h.sum[a];
    }
    res->bad = h.bad;
    return cudaGetLastError();
}

// Morton order of n points: returns the permutation (device, caller frees).
cudaError_t morton_order(const float *x, int64_t n, const BoxResult &bx, cudaStream_t s, int **order_out) {
    unsigned *code = nullptr, *code2 = nullptr;
    int *idx = nullptr, *idx2 = nullptr;
    void *tmp = nullptr;
    size_t tb = 0;
    cudaError_t e = cudaMallocAsync(&code, 4 * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&code2, 4 * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&idx, 4 * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&idx2, 4 * n, s);
    if (e == cudaSuccess) {
        float3 lo = make_float3(bx.lo[0], bx.lo[1], bx.lo[2]);
        float ext[3];
        for (int a = 0; a < 3; ++a) ext[a] = bx.hi[a] - bx.lo[a];
        float3 inv = make_float3(ext[0] > 0 ? 1.0f / ext[0] : 0.0f, ext[1] > 0 ? 1.0f / ext[1] : 0.0f,
                                 ext[2] > 0 ? 1.0f / ext[2] : 0.0f);
        k_morton<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, lo, inv, code, idx);
        counters().launches += 1;
        e = cub::DeviceRadixSort::SortPairs(nullptr, tb, code, code2, idx, idx2, (int)n, 0, 30, s);
    }
    if (e == cudaSuccess) e = cudaMallocAsync(&tmp, tb > 0 ? tb : 16, s);
    if (e == cudaSuccess) {
        // The sort is captured into a graph so its kernel launches can be counted exactly.
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t es = cub::DeviceRadixSort::SortPairs(tmp, tb, code, code2, idx, idx2, (int)n, 0, 30, s);
            e = cudaStreamEndCapture(s, &g);
            if (es != cudaSuccess) e = es;
        }
        if (e == cudaSuccess) {
            size_t nn = 0;
            cudaGraphGetNodes(g, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
            for (size_t k = 0; k < nn; ++k) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nodes[k], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                    counters().launches += 1;
            }
            e = cudaGraphInstantiate(&ge, g, 0);
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
    }
    if (tmp) cudaFreeAsync(tmp, s);
    if (code) cudaFreeAsync(code, s);
    if (code2) cudaFreeAsync(code2, s);
    if (idx) cudaFreeAsync(idx, s);
    if (e != cudaSuccess) {
        if (idx2) cudaFreeAsync(idx2, s);
        return e;
    }
    *order_out = idx2;
    return cudaGetLastError();
}

}  // namespace

cudaError_t build_target(const float *q_dev, const float *n_dev, int64_t n, cudaStream_t s, TargetDev *t,
                         int *bad_input) {
    BoxResult bx;
    cudaError_t e = reduce_box(q_dev, n_dev, n, s, &bx);
    if (e != cudaSuccess) return e;
    *bad_input = bx.bad;
    if (bx.bad) return cudaSuccess;
    t->n = n;
    t->has_normals = n_dev != nullptr;
    for (int a = 0; a < 3; ++a) {
        t->lo[a] = bx.lo[a];
        t->hi[a] = bx.hi[a];
        t->centroid[a] = bx.sum[a] / (double)n;
    }
    const int64_t buckets = (n + kLeaf - 1) / kLeaf;
    int L = 1;
    while (L < buckets) L *= 2;
    t->L = L;
    t->E_Q = -1.0;
    t->H_Q = -1.0;
    int *order = nullptr;
    e = morton_order(q_dev, n, bx, s, &order);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&t->pts, sizeof(float4) * n);
    if (e == cudaSuccess && n_dev) e = cudaMalloc(&t->nrm, sizeof(float4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&t->nodes, sizeof(float4) * 8 * (size_t)L);
    if (e == cudaSuccess) {
        t->obb = t->nodes + 4 * (size_t)L;
        k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q_dev, n_dev, order, n, t->pts, t->nrm);
        k_leaf_boxes<<<(L + 255) / 256, 256, 0, s>>>(t->pts, n, L, t->nodes);
        k_leaf_obb<<<(L + 127) / 128, 128, 0, s>>>(t->pts, n, L, t->obb);
        counters().launches += 3;
        for (int first = L / 2; first >= 1; first /= 2) {
            k_level_boxes<<<(first + 255) / 256, 256, 0, s>>>(t->nodes, first, first);
            counters().launches += 1;
        }
        e = cudaGetLastError();
    }
    cudaFreeAsync(order, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

// FP16 storage of the target: each point as half-precision offsets in
// [0, 1] of its bucket's bounding box (a degenerate box axis stores 0), so a
// decoded point lo + u (hi - lo) stays inside the box the tree tests.
__global__ void k_encode16(const float4 *__restrict__ pts, const float4 *__restrict__ nodes, int n, int L,
                           ushort4 *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float4 p = pts[j];
    const int leaf = L + j / kLeaf;
    const float4 lo = nodes[2 * leaf], hi = nodes[2 * leaf + 1];
    const float ex = hi.x - lo.x, ey = hi.y - lo.y, ez = hi.z - lo.z;
    const float ux = ex > 0.0f ? fminf(fmaxf((p.x - lo.x) / ex, 0.0f), 1.0f) : 0.0f;
    const float uy = ey > 0.0f ? fminf(fmaxf((p.y - lo.y) / ey, 0.0f), 1.0f) : 0.0f;
    const float uz = ez > 0.0f ? fminf(fmaxf((p.z - lo.z) / ez, 0.0f), 1.0f) : 0.0f;
    out[j] = make_ushort4(__half_as_ushort(__float2half_rn(ux)), __half_as_ushort(__float2half_rn(uy)),
                          __half_as_ushort(__float2half_rn(uz)), 0);
}

cudaError_t build_fp16_storage(TargetDev *t, cudaStream_t s) {
    if (t->pts16) return cudaSuccess;
    ushort4 *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(ushort4) * (size_t)t->n);
    if (e != cudaSuccess) return e;
    k_encode16<<<(unsigned)((t->n + 255) / 256), 256, 0, s>>>(t->pts, t->nodes, (int)t->n, t->L, p);
    counters().launches += 1;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(p);
        return e;
    }
    t->pts16 = p;
    return cudaSuccess;
}

cudaError_t launch_median(const double *v, int n, void *scratch, double *out_dev, cudaStream_t s) {
    static_assert(sizeof(MedianState) <= (size_t)kMedianScratchBytes, "median scratch");
    MedianState *mst = static_cast<MedianState *>(scratch);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned mblocks = (unsigned)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)(sms > 0 ? sms : 152) * 4);
    k_median_init<<<1, 256, 0, s>>>(mst, n);
    for (int shift = 56; shift >= 0; shift -= 8) {
        k_median_hist<<<mblocks, 256, 0, s>>>(v, n, mst, shift);
        k_median_pick<<<1, 64, 0, s>>>(mst, shift, out_dev);
    }
    counters().launches += 17;
    return cudaGetLastError();
}

cudaError_t target_nu_stats(TargetDev *t, cudaStream_t s) {
    if (t->E_Q >= 0.0 && (!t->has_normals || t->H_Q >= 0.0)) return cudaSuccess;
    if (t->n < 7) {   // fewer than six neighbours: statistic undefined, use 0 (clamped later)
        t->E_Q = 0.0;
        t->H_Q = 0.0;
        return cudaSuccess;
    }
    double *sd = nullptr, *sh = nullptr, *out = nullptr;
    MedianState *mst = nullptr;
    cudaError_t e = cudaMallocAsync(&sd, sizeof(double) * t->n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&mst, sizeof(MedianState), s);
    if (e == cudaSuccess && t->has_normals) e = cudaMallocAsync(&sh, sizeof(double) * t->n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&out, 3 * sizeof(double), s);
    int *flag = reinterpret_cast<int *>(out + 2);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, 3 * sizeof(double), s);
    if (e == cudaSuccess) {
        const Index ix = make_index(*t);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t blocks = std::min<int64_t>((t->n + kKnnBlock / 32 - 1) / (kKnnBlock / 32),
                                                 (int64_t)(sms > 0 ? sms : 152) * 16);
        if (t->L >= 4) {
            const int64_t tiles = (t->n + 31) / 32;
            const int64_t tblocks = std::min<int64_t>((tiles + kKnnBlock / 32 - 1) / (kKnnBlock / 32),
                                                      (int64_t)(sms > 0 ? sms : 152) * 16);
            k_knn6_tile<<<(unsigned)tblocks, kKnnBlock, 0, s>>>(ix, sd, sh, flag);
        } else {
            k_knn6_stats<<<(unsigned)blocks, kKnnBlock, 0, s>>>(ix, sd, sh, flag);
        }
        counters().launches += 1;
        for (int which = 0; which < (sh ? 2 : 1); ++which)
            if (e == cudaSuccess) e = launch_median(which ? sh : sd, (int)t->n, mst, out + which, s);
        double h[3] = {0.0, 0.0, 0.0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
        counters().d2h += 3 * sizeof(double);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        int overflow = 0;
        std::memcpy(&overflow, &h[2], sizeof(int));
        if (e == cudaSuccess && overflow) e = cudaErrorLaunchOutOfResources;   // search stack: never expected
        if (e == cudaSuccess) {
            t->E_Q = h[0];
            t->H_Q = sh ? h[1] : -1.0;
        }
    }
    if (sd) cudaFreeAsync(sd, s);
    if (sh) cudaFreeAsync(sh, s);
    if (out) cudaFreeAsync(out, s);
    if (mst) cudaFreeAsync(mst, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t estimate_normals(const TargetDev *t, int k, const double viewpoint[3], float *out_dev, cudaStream_t s,
                             int *overflow_out) {
    const int K = (int)std::min<int64_t>(k, t->n);
    double *cov = nullptr;
    int *flag = nullptr;
    cudaError_t e = cudaMallocAsync(&cov, sizeof(double) * 6 * (size_t)t->n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&flag, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        const Index ix = make_index(*t);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t blocks = std::min<int64_t>((t->n + kKnnBlock / 32 - 1) / (kKnnBlock / 32),
                                                 (int64_t)(sms > 0 ? sms : 152) * 16);
        k_knn_cov<<<(unsigned)blocks, kKnnBlock, 0, s>>>(ix, K, cov, flag);
        k_normal_from_cov<<<(unsigned)((t->n + 255) / 256), 256, 0, s>>>(ix, cov, viewpoint[0], viewpoint[1],
                                                                         viewpoint[2], out_dev);
        counters().launches += 2;
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    counters().d2h += sizeof(int);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (cov) cudaFreeAsync(cov, s);
    if (flag) cudaFreeAsync(flag, s);
    *overflow_out = h;
    return e;
}

cudaError_t prepare_source(const float *p_dev, int64_t m, cudaStream_t s, float4 *src_out, float lo[3],
                           float hi[3], int *bad_input, const float *n_dev, float4 *nrm_out) {
    BoxResult bx;
    cudaError_t e = reduce_box(p_dev, n_dev, m, s, &bx, 1);   // a zero source normal: no normal at that point
    if (e != cudaSuccess) return e;
    *bad_input = bx.bad;
    if (bx.bad) return cudaSuccess;
    for (int a = 0; a < 3; ++a) {
        lo[a] = bx.lo[a];
        hi[a] = bx.hi[a];
    }
    int *order = nullptr;
    e = morton_order(p_dev, m, bx, s, &order);
    if (e != cudaSuccess) return e;
    k_gather<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p_dev, n_dev, order, m, src_out, nrm_out);
    counters().launches += 1;
    e = cudaGetLastError();
    cudaFreeAsync(order, s);
    return e;
}

}  // namespace fricp
