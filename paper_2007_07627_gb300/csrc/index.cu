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
#include <vector>

#include "fricp_internal.cuh"
#include "select.cuh"

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
                              BoxPartial *out) {
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
            if (!(fabs(l2 - 1.0) <= 2e-3)) bad = 1;
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
__global__ void k_knn6_stats(Index ix, double *__restrict__ stat_d, double *__restrict__ stat_h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ix.n) return;
    const float4 qi = ix.pts[i];
    const double x0 = qi.x, x1 = qi.y, x2 = qi.z;
    double bd[6];
    int bo[6], bj[6];
    for (int s = 0; s < 6; ++s) {
        bd[s] = INFINITY;
        bo[s] = 0x7fffffff;
        bj[s] = -1;
    }
    int stk[kStack];
    double stkd[kStack];
    int sp = 0, node = 1;
    for (;;) {
        if (node < ix.L) {
            const float4 *b = ix.nodes + 4 * node;
            double d[2];
            for (int c = 0; c < 2; ++c) {
                const float4 lo = b[2 * c], hi = b[2 * c + 1];
                const double g0 = fmax(fmax((double)lo.x - x0, x0 - (double)hi.x), 0.0);
                const double g1 = fmax(fmax((double)lo.y - x1, x1 - (double)hi.y), 0.0);
                const double g2 = fmax(fmax((double)lo.z - x2, x2 - (double)hi.z), 0.0);
                d[c] = g0 * g0 + g1 * g1 + g2 * g2;
            }
            int c0 = 2 * node, c1 = c0 + 1;
            double d0 = d[0], d1 = d[1];
            if (d1 < d0) {
                const double t = d0; d0 = d1; d1 = t;
                const int tc = c0; c0 = c1; c1 = tc;
            }
            if (d0 * (1.0 - 1e-12) <= bd[5]) {
                if (d1 * (1.0 - 1e-12) <= bd[5]) {
                    stk[sp] = c1;
                    stkd[sp] = d1;
                    ++sp;
                }
                node = c0;
                continue;
            }
        } else {
            const int beg = (node - ix.L) * kLeaf;
            const int end = min(beg + kLeaf, ix.n);
            for (int j = beg; j < end; ++j) {
                if (j == i) continue;
                const float4 q = ix.pts[j];
                const double a = (double)q.x - x0, b = (double)q.y - x1, c = (double)q.z - x2;
                const double d = a * a + b * b + c * c;
                const int o = __float_as_int(q.w);
                if (d < bd[5] || (d == bd[5] && o < bo[5])) {
                    int s = 5;
                    while (s > 0 && (bd[s - 1] > d || (bd[s - 1] == d && bo[s - 1] > o))) {
                        bd[s] = bd[s - 1];
                        bo[s] = bo[s - 1];
                        bj[s] = bj[s - 1];
                        --s;
                    }
                    bd[s] = d;
                    bo[s] = o;
                    bj[s] = j;
                }
            }
        }
        node = 0;
        while (sp > 0) {
            --sp;
            if (stkd[sp] * (1.0 - 1e-12) <= bd[5]) {
                node = stk[sp];
                break;
            }
        }
        if (node == 0) break;
    }
    stat_d[i] = 0.5 * (sqrt(bd[2]) + sqrt(bd[3]));
    if (stat_h != nullptr) {
        const float4 ni = ix.nrm[i];
        double h[6];
        for (int s = 0; s < 6; ++s) {
            if (bj[s] < 0) {
                h[s] = INFINITY;
                continue;
            }
            const float4 q = ix.pts[bj[s]];
            h[s] = fabs(((double)q.x - x0) * ni.x + ((double)q.y - x1) * ni.y + ((double)q.z - x2) * ni.z);
        }
        for (int a = 1; a < 6; ++a) {   // insertion sort of six values
            const double v = h[a];
            int b = a - 1;
            while (b >= 0 && h[b] > v) {
                h[b + 1] = h[b];
                --b;
            }
            h[b + 1] = v;
        }
        stat_h[i] = 0.5 * (h[2] + h[3]);
    }
}

__global__ void k_median(const double *v, int n, double *out) {
    const double a = block_kth(v, n, (n - 1) / 2);
    const double b = (n % 2) ? a : block_kth(v, n, n / 2);
    if (threadIdx.x == 0) *out = 0.5 * (a + b);
}

struct BoxResult {
    float lo[3], hi[3];
    double sum[3];
    int bad;
};

cudaError_t reduce_box(const float *x, const float *nrm, int64_t n, cudaStream_t s, BoxResult *res) {
    int nb = (int)std::min<int64_t>((n + kRedBlock - 1) / kRedBlock, 1024);
    if (nb < 1) nb = 1;
    BoxPartial *parts = nullptr;
    cudaError_t e = cudaMallocAsync(&parts, sizeof(BoxPartial) * (nb + 1), s);
    if (e != cudaSuccess) return e;
    k_box_partial<<<nb, kRedBlock, 0, s>>>(x, nrm, n, parts);
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
    if (e == cudaSuccess) e = cudaMalloc(&t->nodes, sizeof(float4) * 4 * (size_t)L);
    if (e == cudaSuccess) {
        k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q_dev, n_dev, order, n, t->pts, t->nrm);
        k_leaf_boxes<<<(L + 255) / 256, 256, 0, s>>>(t->pts, n, L, t->nodes);
        counters().launches += 2;
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

cudaError_t target_nu_stats(TargetDev *t, cudaStream_t s) {
    if (t->E_Q >= 0.0 && (!t->has_normals || t->H_Q >= 0.0)) return cudaSuccess;
    if (t->n < 7) {   // fewer than six neighbours: statistic undefined, use 0 (clamped later)
        t->E_Q = 0.0;
        t->H_Q = 0.0;
        return cudaSuccess;
    }
    double *sd = nullptr, *sh = nullptr, *out = nullptr;
    cudaError_t e = cudaMallocAsync(&sd, sizeof(double) * t->n, s);
    if (e == cudaSuccess && t->has_normals) e = cudaMallocAsync(&sh, sizeof(double) * t->n, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&out, 2 * sizeof(double), s);
    if (e == cudaSuccess) {
        const Index ix = make_index(*t);
        k_knn6_stats<<<(unsigned)((t->n + 127) / 128), 128, 0, s>>>(ix, sd, sh);
        k_median<<<1, 1024, 0, s>>>(sd, (int)t->n, out);
        counters().launches += 2;
        if (sh) {
            k_median<<<1, 1024, 0, s>>>(sh, (int)t->n, out + 1);
            counters().launches += 1;
        }
        double h[2] = {0.0, 0.0};
        e = cudaMemcpyAsync(h, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
        counters().d2h += 2 * sizeof(double);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) {
            t->E_Q = h[0];
            t->H_Q = sh ? h[1] : -1.0;
        }
    }
    if (sd) cudaFreeAsync(sd, s);
    if (sh) cudaFreeAsync(sh, s);
    if (out) cudaFreeAsync(out, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t prepare_source(const float *p_dev, int64_t m, cudaStream_t s, float4 *src_out, float lo[3],
                           float hi[3], int *bad_input) {
    BoxResult bx;
    cudaError_t e = reduce_box(p_dev, nullptr, m, s, &bx);
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
    k_gather<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p_dev, nullptr, order, m, src_out, nullptr);
    counters().launches += 1;
    e = cudaGetLastError();
    cudaFreeAsync(order, s);
    return e;
}

}  // namespace fricp
