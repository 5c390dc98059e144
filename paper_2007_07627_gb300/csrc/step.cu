// One device step = one correspondence pass of Alg. 1 / Alg. 2 plus the
// decision that follows it, in two kernels:
//   k_nn     FP64 transform (Sec. 3, x = R p + t), warm start from the previous
//            correspondence, exact closest target point (Eq. 3), one warp per
//            query (warp_nn);
//   k_accum  residual, Welsch weight and energy term (Eq. 10, Eq. 12,
//                Eq. 16) and each point's share of the alignment sums; each block
//                reduces its tile into one FP64 record (fixed shuffle tree, no
//                atomics); the last block reduces all records in a fixed order
//                and runs solver_step() on one thread, so the iteration never
//                leaves the device.
#include "fricp_internal.cuh"
#include "select.cuh"
#include "solver.cuh"

namespace fricp {

namespace {

// Block reduction of K FP64 values per thread through a shared-memory tree
// (fixed order). A warp-shuffle tree would run every add on all 32 lanes; here
// each level runs only the adds it needs, which matters with few FP64 units.
// The upper half of the block folds into the lower half first, so the buffer
// holds K x kBlock/2 doubles.
template <int K>
__device__ __forceinline__ void block_reduce_store(double (&acc)[K], double *out) {
    constexpr int H = kBlock / 2;
    __shared__ double red[K * H];
    if (threadIdx.x >= H) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * H + threadIdx.x - H] = acc[k];
    }
    __syncthreads();
    if (threadIdx.x < H) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * H + threadIdx.x] += acc[k];
    }
    __syncthreads();
    for (int s = H / 2; s > 0; s >>= 1) {
        for (int e = threadIdx.x; e < K * s; e += kBlock) {
            const int k = e / s, t = e - k * s;
            red[k * H + t] += red[k * H + t + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < K) out[threadIdx.x] = red[threadIdx.x * H];
}

// Fixed-order reduction of the tile records: warp w owns columns w, w+8, ...;
// lane l sums rows l, l+32, ... and a shuffle tree finishes the column.
template <int K>
__device__ __forceinline__ void reduce_tiles(const double *partial, int ntiles, double *S) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = wid; k < K; k += kBlock / 32) {
        double v = 0.0;
        for (int r = lane; r < ntiles; r += 32) v += __ldcg(partial + (size_t)r * K + k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) S[k] = v;
    }
    __syncthreads();
}

// Step state every kernel of a step reads first (thread 0 loads, block shares).
struct StepHead {
    double R[9], t[3], c[3];
    double scale, inv2nu2;
    float Rh[9], Rl[9], th[3], tl[3];   // float splits of R and t for the search
    float cut2;
    int phase, done, welsch, M;
};

__device__ __forceinline__ void load_head(const PairState *st, StepHead &h) {
    h.done = st->done;
    h.phase = st->phase;
    h.welsch = st->variant != FRICP_P2P_AA;
    h.M = st->M;
    for (int i = 0; i < 9; ++i) h.R[i] = st->Re[i];
    for (int r = 0; r < 3; ++r) {
        h.t[r] = st->te[r];
        h.c[r] = st->c[r];
    }
    h.scale = st->s;
    h.inv2nu2 = st->nu > 0.0 ? 1.0 / (2.0 * st->nu * st->nu) : 0.0;
    for (int i = 0; i < 9; ++i) split_double(h.R[i], h.Rh[i], h.Rl[i]);
    for (int r = 0; r < 3; ++r) split_double(h.t[r], h.th[r], h.tl[r]);
    // Welsch cap radius in caller units: (d_n / s)^2 with d_n^2 / (2 nu^2) = kWelschCut
    const double cut2 = st->nu > 0.0 ? kWelschCut * 2.0 * st->nu * st->nu / (st->s * st->s) : 0.0;
    h.cut2 = (cut2 > 0.0 && cut2 < 3.0e38) ? (float)(cut2 * (1.0 + 1e-5)) : __int_as_float(0x7f800000);
}

__device__ __forceinline__ void transform_point(const StepHead &h, float4 p, double x[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        x[r] = fma(h.R[3 * r], (double)p.x, fma(h.R[3 * r + 1], (double)p.y, fma(h.R[3 * r + 2], (double)p.z, h.t[r])));
}

// Start a query: FP64 transform, warm start from the previous correspondence,
// and (Welsch point-to-point, after the nu_max pass) the exact weight cap.
template <int VAR>
__device__ __forceinline__ void start_query(const StepArgs &a, const StepHead &h, int i, NNLane &q, bool &cold) {
    float xh[3], xl[3];
    df_transform(h.Rh, h.Rl, h.th, h.tl, __ldg(a.src + i), xh, xl);
    nn_init(q, xh, xl);
    const int j0 = a.prev[i];
    cold = j0 < 0;
    if (!cold) nn_seed(q, __ldg(a.ix.pts + j0), j0);
    // Welsch point-to-point: a point farther than the cap has weight exp(-a) = 0.0
    // and psi = 1.0 exactly for every candidate that far, so the search radius is
    // capped there (the sums are bit-identical).
    if (VAR == 0 && h.welsch && h.phase != PH_INIT && h.cut2 < q.bestf) {
        q.bestf = h.cut2;
        cold = false;
    }
}

// Search kernel: persistent warps walk the Morton-ordered queries; each query
// is searched by a whole warp (warp_nn). Writes prev[i] = this pass's
// correspondence (the next pass's warm start).
template <int VAR>
__global__ void __launch_bounds__(kBlock) k_nn(StepArgs a) {
    __shared__ StepHead h;
    __shared__ int s_stk[kBlock / 32][kWarpStack];
    if (threadIdx.x == 0) load_head(a.st, h);
    __syncthreads();
    if (h.done) return;
    const int lane = threadIdx.x & 31;
    const int wpb = kBlock / 32;
    int *stk = s_stk[threadIdx.x >> 5];
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < h.M; i += gridDim.x * wpb) {
        NNLane q;   // every lane sets up the same query (float arithmetic, broadcast loads)
        bool cold;
        start_query<VAR>(a, h, i, q, cold);
        if (!warp_nn(a.ix, q, stk, q.best_j >= 0 ? q.best_j / kLeaf : -1)) {
            if (lane == 0) a.st->status = FRICP_ECUDA;   // stack overflow: never expected
            q.best_j = 0;
        }
        if (lane == 0) a.prev[i] = q.best_j < 0 ? 0 : q.best_j;   // -1 only if nothing lies inside the cap
        __syncwarp();
    }
}

// Kernel C: per-point FP64 terms at this pass's correspondences, tile records,
// and in the last block the fixed-order reduction and the solver step.
template <int VAR>
__global__ void __launch_bounds__(kBlock) k_accum(StepArgs a) {
    constexpr int K = VAR ? kSumsP2PL : kSumsP2P;
    PairState *st = a.st;
    __shared__ StepHead h;
    __shared__ double sS[K];
    __shared__ int s_last;
    if (threadIdx.x == 0) load_head(st, h);
    __syncthreads();
    if (h.done) return;

    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i < h.M) {
        const float4 p = __ldg(a.src + i);
        double x[3];
        transform_point(h, p, x);
        const int j = a.prev[i];
        const float4 q = __ldg(a.ix.pts + j);
        const double dx = x[0] - (double)q.x, dy = x[1] - (double)q.y, dz = x[2] - (double)q.z;
        const double s = h.scale;
        const double pt[3] = {(double)p.x - h.c[0], (double)p.y - h.c[1], (double)p.z - h.c[2]};
        if (VAR == 0) {
            const double d2n = s * s * (dx * dx + dy * dy + dz * dz);
            double w, psi;
            if (h.welsch) {
                w = exp(-d2n * h.inv2nu2);
                psi = 1.0 - w;
            } else {
                w = 1.0;
                psi = d2n;
            }
            if (h.phase == PH_INIT) a.resid[i] = sqrt(d2n);
            const double qt[3] = {(double)q.x - h.c[0], (double)q.y - h.c[1], (double)q.z - h.c[2]};
            acc[0] = w;
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                acc[1 + u] = w * pt[u];
                acc[4 + u] = w * qt[u];
            }
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v) acc[7 + 3 * u + v] = acc[1 + u] * qt[v];
            acc[16] = psi;
        } else {
            const float4 nv = __ldg(a.ix.nrm + j);
            const double n0 = nv.x, n1 = nv.y, n2 = nv.z;
            const double hh = s * (dx * n0 + dy * n1 + dz * n2);
            if (h.phase == PH_INIT) a.resid[i] = fabs(hh);
            const double g = exp(-hh * hh * h.inv2nu2);
            // y = R p~ in normalised units; z = [y x n; n]
            double y[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) y[r] = s * (h.R[3 * r] * pt[0] + h.R[3 * r + 1] * pt[1] + h.R[3 * r + 2] * pt[2]);
            const double z[6] = {y[1] * n2 - y[2] * n1, y[2] * n0 - y[0] * n2, y[0] * n1 - y[1] * n0, n0, n1, n2};
            int t = 0;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const double gz = g * z[r];
#pragma unroll
                for (int c = r; c < 6; ++c) acc[t++] = gz * z[c];
                acc[21 + r] = gz * hh;
            }
            acc[27] = 1.0 - g;
        }
    }
    block_reduce_store<K>(acc, a.partial + (size_t)blockIdx.x * K);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&st->counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    reduce_tiles<K>(a.partial, gridDim.x, sS);
    if (h.phase == PH_INIT) {
        const int n = h.M;
        const double lo = block_kth(a.resid, n, (n - 1) / 2);
        const double hi = (n % 2) ? lo : block_kth(a.resid, n, n / 2);
        if (threadIdx.x == 0) {
            st->device_steps++;
            if (st->eval_counts) st->corr_passes++;
            start_after_init(st, 0.5 * (lo + hi));
        }
    } else if (threadIdx.x == 0) {
        solver_step(st, sS, a.trace);
    }
    if (threadIdx.x == 0) st->counter = 0u;
}

// Correspondence step alone: index (original order) and FP64 squared distance.
__global__ void __launch_bounds__(128) k_closest(Index ix, const float *__restrict__ p, int64_t m,
                                                 const double *__restrict__ T, int64_t *__restrict__ idx,
                                                 double *__restrict__ d2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < m;
    if (active) {
        float Rh[9], Rl[9], th[3], tl[3], xh[3], xl[3];
        for (int k = 0; k < 9; ++k) split_double(T[k], Rh[k], Rl[k]);
        for (int r = 0; r < 3; ++r) split_double(T[9 + r], th[r], tl[r]);
        const float4 pp = make_float4(p[3 * i], p[3 * i + 1], p[3 * i + 2], 0.0f);
        df_transform(Rh, Rl, th, tl, pp, xh, xl);
        NNLane q;
        nn_init(q, xh, xl);
        nn_thread(ix, q);
        if (q.best_j < 0) q.best_j = 0;   // only for a non-finite x
        const float4 qq = __ldg(ix.pts + q.best_j);
        double x[3];
        for (int r = 0; r < 3; ++r) x[r] = fma(T[3 * r], (double)pp.x, fma(T[3 * r + 1], (double)pp.y, fma(T[3 * r + 2], (double)pp.z, T[9 + r])));
        const double dx = x[0] - (double)qq.x, dy = x[1] - (double)qq.y, dz = x[2] - (double)qq.z;
        idx[i] = __float_as_int(qq.w);
        d2[i] = dx * dx + dy * dy + dz * dz;
    }
}

// Single-evaluation set-up for fricp_eval_pass: T is normalised (R, t).
__global__ void k_setup_eval(PairState *st, const double *T) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double Tn[12];
    for (int i = 0; i < 12; ++i) Tn[i] = T[i];
    if (st->variant == FRICP_P2PL_WELSCH_AA) {
        double xi[6];
        se3_log(Tn, xi);
        request_eval_xi(st, xi, 1);
    } else {
        request_eval_T(st, Tn, 1);
    }
    st->phase = PH_EVAL;
}

}  // namespace

// Blocks of the search kernel (persistent warps): enough to fill every SM.
int nn_blocks(int M) {
    static int nb = 0;
    if (nb == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nn<0>, kBlock, 0);
        nb = (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
    }
    const int need = (M + kBlock / 32 - 1) / (kBlock / 32);
    return need < nb ? need : nb;
}

cudaError_t launch_step(const StepArgs &a, int variant, int ntiles, cudaStream_t s) {
    const int nb = nn_blocks(ntiles * kBlock);
    if (variant == FRICP_P2PL_WELSCH_AA) {
        k_nn<1><<<nb, kBlock, 0, s>>>(a);
        k_accum<1><<<ntiles, kBlock, 0, s>>>(a);
    } else {
        k_nn<0><<<nb, kBlock, 0, s>>>(a);
        k_accum<0><<<ntiles, kBlock, 0, s>>>(a);
    }
    counters().launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_closest(const TargetDev *t, const float *p_dev, int64_t m, const double T[12], int64_t *idx,
                           double *d2, cudaStream_t s) {
    double *dT = nullptr;
    cudaError_t e = cudaMallocAsync(&dT, 12 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dT, T, 12 * sizeof(double), cudaMemcpyHostToDevice, s);
    counters().h2d += 12 * sizeof(double);
    if (e == cudaSuccess) {
        const Index ix = make_index(*t);
        k_closest<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(ix, p_dev, m, dT, idx, d2);
        counters().launches += 1;
        e = cudaGetLastError();
    }
    cudaFreeAsync(dT, s);
    return e;
}

cudaError_t launch_setup_eval_xi(PairState *st, const double *T_normalized12, cudaStream_t s) {
    k_setup_eval<<<1, 32, 0, s>>>(st, T_normalized12);
    counters().launches += 1;
    return cudaGetLastError();
}

}  // namespace fricp
