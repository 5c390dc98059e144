// Device code shared by the single-registration step (step.cu) and the batched
// step (batch.cu): the per-step head of a registration, the start of a query,
// each point's share of the alignment sums, the block and tile reductions and
// the work of the block that completes a registration's pass. Both paths run
// exactly this arithmetic in this order, so a registration gives the same bits
// alone and inside a batch.
#pragma once

#include "fricp_internal.cuh"
#include "select.cuh"
#include "solver.cuh"

namespace fricp {
namespace {

// Shared buffer of block_reduce_store: K x kBlock/2 doubles.
constexpr int kRedHalf = kBlock / 2;

// Block reduction of K FP64 values per thread through a shared-memory tree
// (fixed order). A warp-shuffle tree would run every add on all 32 lanes; here
// each level runs only the adds it needs, which matters with few FP64 units.
// The upper half of the block folds into the lower half first. `red` holds
// K * kRedHalf doubles of shared memory.
template <int K>
__device__ __forceinline__ void block_reduce_store(double (&acc)[K], double *out, double *red) {
    constexpr int H = kRedHalf;
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
    __syncthreads();   // `red` may be reused right away
}

// Fixed-order reduction of the tile records: thread t < G K (G = kBlock / K row
// groups) sums column t mod K over rows g, g + G, g + 2 G, ... (g = t / K) in
// order, eight loads in flight; the G partial sums of a column are then added
// in group order. `red` holds kBlock doubles of shared memory.
template <int K>
__device__ __forceinline__ void reduce_tiles(const double *partial, int ntiles, double *S, double *red) {
    constexpr int G = kBlock / K;
    const int t = threadIdx.x;
    if (t < G * K) {
        const int k = t % K, g = t / K;
        double v = 0.0;
        int r = g;
        for (; r + G * 7 < ntiles; r += G * 8) {
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __ldcg(partial + (size_t)(r + G * u) * K + k);
#pragma unroll
            for (int u = 0; u < 8; ++u) v += x[u];
        }
        for (; r < ntiles; r += G) v += __ldcg(partial + (size_t)r * K + k);
        red[t] = v;
    }
    __syncthreads();
    if (t < K) {
        double v = red[t];
        for (int g = 1; g < G; ++g) v += red[g * K + t];
        S[t] = v;
    }
    __syncthreads();
}

// Step state every kernel of a step reads first.
struct StepHead {
    double R[9], t[3], c[3];
    double scale, inv2nu2;
    float Rh[9], Rl[9], th[3], tl[3];   // float splits of R and t for the search
    float cut2;
    int phase, done, welsch, M, variant, prec;
};

__device__ __forceinline__ void load_head(const PairState *st, StepHead &h) {
    h.done = st->done;
    h.phase = st->phase;
    h.variant = st->variant;
    h.prec = st->prec;
    h.welsch = fricp::variant_robust(st->variant);
    h.M = st->M;
    for (int i = 0; i < 9; ++i) h.R[i] = st->Re[i];
    for (int r = 0; r < 3; ++r) {
        h.t[r] = st->te[r];
        h.c[r] = st->c[r];
    }
    h.scale = st->s;
    h.inv2nu2 = st->hinv2nu2;   // the derived values were set with Re, te and nu (set_head_cache)
    for (int i = 0; i < 9; ++i) {
        h.Rh[i] = st->hRh[i];
        h.Rl[i] = st->hRl[i];
    }
    for (int r = 0; r < 3; ++r) {
        h.th[r] = st->hth[r];
        h.tl[r] = st->htl[r];
    }
    h.cut2 = st->hcut2;
}

__device__ __forceinline__ void transform_point(const StepHead &h, float4 p, double x[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        x[r] = fma(h.R[3 * r], (double)p.x, fma(h.R[3 * r + 1], (double)p.y, fma(h.R[3 * r + 2], (double)p.z, h.t[r])));
}

// Start a query: double-float transform, warm start from the previous
// correspondence, and (Welsch point-to-point after the nu_max pass) the exact
// weight cap: a point farther than the cap has weight exp(-a) = 0.0 and
// psi = 1.0 exactly for every candidate that far, so the search radius is capped
// there (the sums are bit-identical).
template <int PREC>
__device__ __forceinline__ void start_query(const Index &ix, const float4 *src, const int *prev, const StepHead &h,
                                            int i, bool p2p, NNLane &q) {
    float xh[3], xl[3];
    const float4 p = __ldg(src + i);
    if (PREC == PREC_FP64) {
        df_transform(h.Rh, h.Rl, h.th, h.tl, p, xh, xl);
    } else {   // float transform with R and t rounded to float
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            xh[r] = fmaf(h.Rh[3 * r], p.x, fmaf(h.Rh[3 * r + 1], p.y, fmaf(h.Rh[3 * r + 2], p.z, h.th[r])));
            xl[r] = 0.0f;
        }
    }
    nn_init(q, xh, xl);
    const int j0 = prev[i];
    if (j0 >= 0) nn_seed<PREC>(q, target_point<PREC>(ix, j0), j0);
    if (p2p && h.welsch && h.phase != PH_INIT && h.cut2 < q.bestf) q.bestf = h.cut2;
}

// One query searched by the whole warp; lane 0 stores the correspondence (the
// next pass's warm start). Returns false on a search-stack overflow.
template <int PREC>
__device__ __forceinline__ bool search_query(const Index &ix, const float4 *src, int *prev, const StepHead &h, int i,
                                             bool p2p, int *stk) {
    NNLane q;   // every lane sets up the same query (float arithmetic, broadcast loads)
    start_query<PREC>(ix, src, prev, h, i, p2p, q);
    const bool ok = warp_nn<PREC>(ix, q, stk, q.best_j >= 0 ? q.best_j / kLeaf : -1);
    if (!ok) q.best_j = 0;
    if ((threadIdx.x & 31) == 0) prev[i] = q.best_j < 0 ? 0 : q.best_j;   // -1 only if nothing lies inside the cap
    __syncwarp();
    return ok;
}

// Two queries per warp (halfwarp_nn): lanes 0-15 search query i, lanes 16-31
// query i + 1 (when `live`); lane 0 of each half stores its correspondence.
// Returns false on a search-stack overflow.
template <int PREC>
__device__ __forceinline__ bool search_pair(const Index &ix, const float4 *src, int *prev, const StepHead &h, int i,
                                            bool live, bool p2p, int *stk_half) {
    NNLane q;
    if (live) {
        start_query<PREC>(ix, src, prev, h, i, p2p, q);
    } else {
        const float z[3] = {0.0f, 0.0f, 0.0f};
        nn_init(q, z, z);
    }
    const bool ok = halfwarp_nn<PREC>(ix, q, stk_half, live && q.best_j >= 0 ? q.best_j / kLeaf : -1, live);
    if (live && (threadIdx.x & 15) == 0) prev[i] = (!ok || q.best_j < 0) ? 0 : q.best_j;
    __syncwarp();
    return ok;
}

// Queries i0 .. i0 + kTileQ - 1 (below i1) as one query tile (tile_nn); the
// queries it sets aside (no warm start: the first pass) are then searched one
// by one by the whole warp (warp_nn). The group head stores each
// correspondence. `wbuf`: kWarpStack ints per warp; `stage`: kRing x 32
// float4. Returns false on a search-stack overflow.
template <int PREC>
__device__ __forceinline__ bool search_tile(const Index &ix, const float4 *src, int *prev, const StepHead &h, int i0,
                                            int i1, bool p2p, int *wbuf, float4 *stage) {
    const int lane = threadIdx.x & 31;
    const int i = i0 + (lane >> 2);
    const bool live = i < i1;
    NNLane q;
    if (live) {
        start_query<PREC>(ix, src, prev, h, i, p2p, q);
    } else {
        const float z[3] = {0.0f, 0.0f, 0.0f};
        nn_init(q, z, z);
    }
    const unsigned aside = tile_nn<PREC>(ix, q, live, wbuf, wbuf + kTileStack, stage);
    if (live && (lane & 3) == 0 && !((aside >> lane) & 1u)) prev[i] = q.best_j;   // warm-started: best_j >= 0
    __syncwarp();
    bool ok = true;
    unsigned heads = aside & 0x11111111u;
    while (heads) {
        const int g = (__ffs(heads) - 1) >> 2;
        heads &= heads - 1u;
        ok = search_query<PREC>(ix, src, prev, h, i0 + g, p2p, wbuf) && ok;
    }
    return ok;
}

// Point i's share of the pass sums at this pass's correspondence:
// Welsch weight and energy term (Eq. 10, Eq. 12, Eq. 16); point-to-point: the
// weighted centroids and cross-covariance terms; point-to-plane: g z z^T, g z h
// and the energy with z = [y x n; n] (App. D). At PH_INIT the residual is kept
// for the nu_max median. PREC_FP64: every term in FP64. PREC_FP32 / PREC_FP16:
// transform, residual, weight and the products in float, widened to FP64 for
// the sums.
template <int VAR, int PREC>
__device__ __forceinline__ void accum_point(const StepHead &h, const Index &ix, const float4 *src, const int *prev,
                                            double *resid, int i, double (&acc)[VAR ? kSumsP2PL : kSumsP2P],
                                            const float4 *src_nrm = nullptr) {
    const float4 p = __ldg(src + i);
    const int j = prev[i];
    const float4 q = target_point<PREC>(ix, j);
    if (PREC != PREC_FP64) {
        float x[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            x[r] = fmaf(h.Rh[3 * r], p.x, fmaf(h.Rh[3 * r + 1], p.y, fmaf(h.Rh[3 * r + 2], p.z, h.th[r])));
        const float dx = x[0] - q.x, dy = x[1] - q.y, dz = x[2] - q.z;
        const float s = (float)h.scale, c0 = (float)h.c[0], c1 = (float)h.c[1], c2 = (float)h.c[2];
        const float i2 = (float)h.inv2nu2;
        const float pt[3] = {p.x - c0, p.y - c1, p.z - c2};
        if (VAR == 0) {
            const float d2n = s * s * fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            float w, psi;
            if (h.welsch) {
                w = expf(-d2n * i2);
                psi = 1.0f - w;
            } else {
                w = 1.0f;
                psi = d2n;
            }
            if (h.phase == PH_INIT) resid[i] = (double)sqrtf(d2n);
            const float qt[3] = {q.x - c0, q.y - c1, q.z - c2};
            acc[0] = w;
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                acc[1 + u] = (double)(w * pt[u]);
                acc[4 + u] = (double)(w * qt[u]);
            }
#pragma unroll
            for (int u = 0; u < 3; ++u)
#pragma unroll
                for (int v = 0; v < 3; ++v) acc[7 + 3 * u + v] = (double)(w * pt[u] * qt[v]);
            acc[16] = psi;
        } else {
            float4 nv = __ldg(ix.nrm + j);
            float rn[3] = {0.0f, 0.0f, 0.0f};
            if (src_nrm != nullptr && fricp::variant_sym(h.variant)) {
                // symmetric objective: the pair's normal is nq + R np (the source normal moved)
                const float4 np = __ldg(src_nrm + i);
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    rn[r] = fmaf(h.Rh[3 * r], np.x, fmaf(h.Rh[3 * r + 1], np.y, h.Rh[3 * r + 2] * np.z));
                nv.x += rn[0];
                nv.y += rn[1];
                nv.z += rn[2];
            }
            const float hh = s * fmaf(dz, nv.z, fmaf(dy, nv.y, dx * nv.x));
            if (h.phase == PH_INIT) resid[i] = (double)fabsf(hh);
            const float g = h.welsch ? expf(-hh * hh * i2) : 1.0f;   // plain point-to-plane: weights 1
            float y[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                y[r] = s * fmaf(h.Rh[3 * r], pt[0], fmaf(h.Rh[3 * r + 1], pt[1], h.Rh[3 * r + 2] * pt[2]));
            // z = [y x n + (R np) x d; n] with d = s (x - q) (the second term: symmetric objective only)
            const float d0 = s * dx, d1 = s * dy, d2 = s * dz;
            const float z[6] = {y[1] * nv.z - y[2] * nv.y + (rn[1] * d2 - rn[2] * d1),
                                y[2] * nv.x - y[0] * nv.z + (rn[2] * d0 - rn[0] * d2),
                                y[0] * nv.y - y[1] * nv.x + (rn[0] * d1 - rn[1] * d0), nv.x, nv.y, nv.z};
            int t = 0;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const float gz = g * z[r];
#pragma unroll
                for (int c = r; c < 6; ++c) acc[t++] = (double)(gz * z[c]);
                acc[21 + r] = (double)(gz * hh);
            }
            acc[27] = h.welsch ? (double)(1.0f - g) : (double)(hh * hh);
        }
        return;
    }
    double x[3];
    transform_point(h, p, x);
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
        if (h.phase == PH_INIT) resid[i] = sqrt(d2n);
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
        const float4 nv = __ldg(ix.nrm + j);
        double n0 = nv.x, n1 = nv.y, n2 = nv.z;
        const bool sym = src_nrm != nullptr && fricp::variant_sym(h.variant);
        double rn[3] = {0.0, 0.0, 0.0};
        if (sym) {   // symmetric objective: the pair's normal is nq + R np (the source normal moved)
            const float4 np = __ldg(src_nrm + i);
#pragma unroll
            for (int r = 0; r < 3; ++r)
                rn[r] = h.R[3 * r] * (double)np.x + h.R[3 * r + 1] * (double)np.y + h.R[3 * r + 2] * (double)np.z;
            n0 += rn[0];
            n1 += rn[1];
            n2 += rn[2];
        }
        const double hh = s * (dx * n0 + dy * n1 + dz * n2);
        if (h.phase == PH_INIT) resid[i] = fabs(hh);
        const double g = h.welsch ? exp(-hh * hh * h.inv2nu2) : 1.0;   // plain point-to-plane: weights 1
        // y = R p~ in normalised units; z = [y x n; n], plus (R np) x d in the rotational part for the
        // symmetric objective (d = s (x - q), the residual vector in normalised units)
        double y[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) y[r] = s * (h.R[3 * r] * pt[0] + h.R[3 * r + 1] * pt[1] + h.R[3 * r + 2] * pt[2]);
        double z[6] = {y[1] * n2 - y[2] * n1, y[2] * n0 - y[0] * n2, y[0] * n1 - y[1] * n0, n0, n1, n2};
        if (sym) {
            const double d0 = s * dx, d1 = s * dy, d2 = s * dz;
            z[0] += rn[1] * d2 - rn[2] * d1;
            z[1] += rn[2] * d0 - rn[0] * d2;
            z[2] += rn[0] * d1 - rn[1] * d0;
        }
        int t = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const double gz = g * z[r];
#pragma unroll
            for (int c = r; c < 6; ++c) acc[t++] = gz * z[c];
            acc[21 + r] = gz * hh;
        }
        acc[27] = h.welsch ? 1.0 - g : hh * hh;
    }
}

// One tile of kBlock points of a registration: per-point terms, then the tile's
// FP64 record at partial[tile * K]. Returns true in every thread of the block
// that completed the registration's pass (the last of its tiles to finish).
template <int VAR, int PREC>
__device__ __forceinline__ bool accum_tile(const StepHead &h, PairState *st, const Index &ix, const float4 *src,
                                           const int *prev, double *resid, double *partial, int tile, int ntiles,
                                           double *red, int *s_last, const float4 *src_nrm = nullptr) {
    constexpr int K = VAR ? kSumsP2PL : kSumsP2P;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const int i = tile * kBlock + threadIdx.x;
    if (i < h.M) accum_point<VAR, PREC>(h, ix, src, prev, resid, i, acc, src_nrm);
    block_reduce_store<K>(acc, partial + (size_t)tile * K, red);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_last = (atomicAdd(&st->counter, 1u) == (unsigned)ntiles - 1u);
    __syncthreads();
    const bool last = *s_last != 0;
    if (last) __threadfence();
    return last;
}

// Work of the block that completed a pass: the fixed-order reduction of the
// tile records, then either the nu_max median (PH_INIT) or one solver step by
// the block's first warp (team scratch: `team_sh`, kTeamScratch doubles of
// shared memory free at this point). Resets the tile counter for the next pass.
template <int K>
__device__ __forceinline__ void finish_pass(const StepHead &h, PairState *st, const double *partial, int ntiles,
                                            const double *resid, double *trace, double *sS, double *team_sh) {
    reduce_tiles<K>(partial, ntiles, sS, team_sh);
    if (h.phase == PH_INIT && st->init_median_ext) {
        // the host selects the median with the whole GPU (launch_median) and
        // then starts the first stage (launch_after_init)
        if (threadIdx.x == 0) {
            st->device_steps++;
            if (st->eval_counts) st->corr_passes++;
            st->counter = 0u;   // the next pass's tile and search tickets start over
            st->nn_next = 0u;
        }
    } else if (h.phase == PH_INIT) {
        const int n = h.M;
        double lo, hi;
        block_median_pair(resid, n, &lo, &hi);
        if (threadIdx.x == 0) {
            st->device_steps++;
            if (st->eval_counts) st->corr_passes++;
            start_after_init(st, 0.5 * (lo + hi));
            st->counter = 0u;   // the next pass's tile and search tickets start over
            st->nn_next = 0u;
        }
    } else if (threadIdx.x < kTeamLanes) {
        solver_step(Team{team_sh}, st, sS, trace);   // resets the tickets in its copy of the state
    }
    __syncthreads();
}

}  // namespace
}  // namespace fricp
