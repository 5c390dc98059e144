// One device step = one correspondence pass of Alg. 1 / Alg. 2 plus the
// decision that follows it, in two kernels:
//   k_nn_tile double-float transform (Sec. 3, x = R p + t), warm start from the
//            previous correspondence, exact closest target point (Eq. 3), one
//            warp per tile of kTileQ Morton-adjacent queries (tile_nn); k_nn,
//            one warp per query (warp_nn), is the alternative search;
//   k_accum  residual, Welsch weight and energy term (Eq. 10, Eq. 12, Eq. 16)
//            and each point's share of the alignment sums in FP64; each block
//            reduces its tile into one record (fixed shared-memory tree, no
//            atomics); the last block reduces all records in a fixed order and
//            runs solver_step() on one warp, so the iteration never leaves
//            the device.
#include "step_common.cuh"

namespace fricp {

namespace {

// Search kernel: persistent warps walk the Morton-ordered queries; each query
// is searched by a whole warp. Writes prev[i] = this pass's correspondence (the
// next pass's warm start).
template <int PREC>
__global__ void __launch_bounds__(kBlock) k_nn(StepArgs a) {
    __shared__ StepHead h;
    __shared__ int s_stk[kBlock / 32][kWarpStack];
    if (threadIdx.x == 0) load_head(a.st, h);
    __syncthreads();
    if (h.done) return;
    const int wpb = kBlock / 32;
    const bool p2p = !fricp::variant_p2pl(h.variant);
    if (p2p && h.welsch && h.phase != PH_INIT) {
        // Welsch cap active: queries beyond it end after a round or two while the
        // others search their neighbourhood, so a pair of queries would wait for
        // the harder one: one query per warp
        int *stk = s_stk[threadIdx.x >> 5];
        for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < h.M; i += gridDim.x * wpb) {
            if (!search_query<PREC>(a.ix, a.src, a.prev, h, i, p2p, stk) && (threadIdx.x & 31) == 0)
                a.st->nn_overflow = 1;   // search-stack overflow: never expected
        }
    } else {
        // similar work per query: two Morton-adjacent queries per warp, one per
        // half; each warp takes the next pair from a counter in the state, so
        // the SMs finish together (each pair's result depends only on the pair)
        int *stk = s_stk[threadIdx.x >> 5] + (threadIdx.x & 16 ? kHalfStack : 0);
        for (;;) {
            unsigned e = 0;
            if ((threadIdx.x & 31) == 0) e = atomicAdd(&a.st->nn_next, 1u);
            e = __shfl_sync(0xffffffffu, e, 0);
            if (2 * (long long)e >= h.M) break;
            const int i = 2 * (int)e + ((threadIdx.x & 16) ? 1 : 0);
            if (!search_pair<PREC>(a.ix, a.src, a.prev, h, i, i < h.M, p2p, stk) && (threadIdx.x & 31) == 0)
                a.st->nn_overflow = 1;   // search-stack overflow: never expected
        }
    }
}

// Search kernel over query tiles: persistent warps take tiles of kTileQ
// Morton-adjacent queries (four lanes per query, search_tile) from a counter
// in the state (the tiles' costs vary with the surface and the outliers they
// hold). Each result depends only on its query, so the order changes no bit.
template <int PREC>
__global__ void __launch_bounds__(kBlock) k_nn_tile(StepArgs a) {
    __shared__ StepHead h;
    __shared__ int s_buf[kBlock / 32][kWarpStack];
    __shared__ __align__(16) float4 s_stage[kBlock / 32][kRing * 32];
    if (threadIdx.x == 0) load_head(a.st, h);
    __syncthreads();
    if (h.done) return;
    const bool p2p = !fricp::variant_p2pl(h.variant);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned e = 0;
        if (lane == 0) e = atomicAdd(&a.st->nn_next, 1u);
        e = __shfl_sync(0xffffffffu, e, 0);
        if ((long long)kTileQ * e >= h.M) break;
        const int i0 = kTileQ * (int)e;
        if (!search_tile<PREC>(a.ix, a.src, a.prev, h, i0, min(i0 + kTileQ, h.M), p2p, s_buf[w], s_stage[w]) &&
            lane == 0)
            a.st->nn_overflow = 1;   // search-stack overflow: never expected
    }
}

// Accumulate kernel: one tile of points per block; the block that completes
// the pass reduces the records and runs the solver step.
template <int VAR, int PREC>
__global__ void __launch_bounds__(kBlock, 3) k_accum(StepArgs a) {
    constexpr int K = VAR ? kSumsP2PL : kSumsP2P;
    __shared__ StepHead h;
    __shared__ double red[K * kRedHalf];
    __shared__ double sS[K];
    __shared__ int s_last;
    if (threadIdx.x == 0) load_head(a.st, h);
    __syncthreads();
    if (h.done) return;
    if (accum_tile<VAR, PREC>(h, a.st, a.ix, a.src, a.prev, a.resid, a.partial, blockIdx.x, gridDim.x, red, &s_last,
                              a.src_nrm))
        finish_pass<K>(h, a.st, a.partial, gridDim.x, a.resid, a.trace, sS, red);
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

// Single-evaluation set-up for fricp_eval_pass: T is normalised (R, t). One warp.
__global__ void __launch_bounds__(32) k_after_init(PairState *st, const double *median) {
    if (threadIdx.x == 0) start_after_init(st, *median);   // nu_max and the first stage, as after a block median
}

__global__ void __launch_bounds__(32) k_setup_eval(PairState *gst, const double *T) {
    __shared__ double sh[kTeamScratch];
    if (threadIdx.x >= kTeamLanes) return;
    const Team tm{sh};
    PairState own;
    load_state(tm, gst, &own);
    PairState *st = &own;
    double Tn[12];
    for (int i = 0; i < 12; ++i) Tn[i] = T[i];
    if (fricp::variant_p2pl(st->variant)) {
        double xi[6];
        log_state_T(tm, Tn, xi);
        request_eval_xi(tm, st, xi, 1);
    } else {
        request_eval_state_T(tm, st, Tn, 1);
    }
    st->phase = PH_EVAL;
    set_head_cache(tm, st);
    store_state(tm, st, gst);
}

}  // namespace

// Blocks of a persistent search kernel: enough to fill every SM at that
// kernel's occupancy, and no more than the work units need (M / per_warp
// queries per warp).
template <typename K>
int persistent_blocks(K kernel, int *cache, int M, int per_warp) {
    if (*cache == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0);
        *cache = (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1);
    }
    const int warps = (M + per_warp - 1) / per_warp;
    const int need = (warps + kBlock / 32 - 1) / (kBlock / 32);
    return need < *cache ? need : *cache;
}

template <int PREC>
void launch_step_prec(const StepArgs &a, int variant, int ntiles, int search, cudaStream_t s, cudaEvent_t mid) {
    static int nb_query = 0, nb_tile = 0;
    if (search == FRICP_SEARCH_QUERY)
        k_nn<PREC><<<persistent_blocks(k_nn<PREC>, &nb_query, ntiles * kBlock, 1), kBlock, 0, s>>>(a);
    else
        k_nn_tile<PREC><<<persistent_blocks(k_nn_tile<PREC>, &nb_tile, ntiles * kBlock, kTileQ), kBlock, 0, s>>>(a);
    if (mid) cudaEventRecord(mid, s);
    if (fricp::variant_p2pl(variant))
        k_accum<1, PREC><<<ntiles, kBlock, 0, s>>>(a);
    else
        k_accum<0, PREC><<<ntiles, kBlock, 0, s>>>(a);
}

cudaError_t launch_step(const StepArgs &a, int variant, int prec, int ntiles, cudaStream_t s, cudaEvent_t mid,
                        int search) {
    if (prec == PREC_FP32)
        launch_step_prec<PREC_FP32>(a, variant, ntiles, search, s, mid);
    else if (prec == PREC_FP16)
        launch_step_prec<PREC_FP16>(a, variant, ntiles, search, s, mid);
    else
        launch_step_prec<PREC_FP64>(a, variant, ntiles, search, s, mid);
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

cudaError_t launch_after_init(PairState *st, const double *median_dev, cudaStream_t s) {
    k_after_init<<<1, 32, 0, s>>>(st, median_dev);
    counters().launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_setup_eval_xi(PairState *st, const double *T_normalized12, cudaStream_t s) {
    k_setup_eval<<<1, 32, 0, s>>>(st, T_normalized12);
    counters().launches += 1;
    return cudaGetLastError();
}

}  // namespace fricp
