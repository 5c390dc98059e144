// The fused step kernel: one correspondence pass of Alg. 1 / Alg. 2 plus the
// decision that follows it, in a single launch.
//
// Each block owns one tile of kBlock sorted source points. Per point (one per
// thread): transform in FP64 (Sec. 3, x = R p + t), exact closest target point
// (Eq. 3), residual, Welsch weight and energy term (Eq. 10, Eq. 12, Eq. 16), and
// that point's contribution to the alignment sums. The block reduces its tile
// into one FP64 record (fixed shuffle tree, no atomics). The last block to
// finish reduces all tile records in a fixed order and runs solver_step() on one
// thread, so the iteration never leaves the device.
#include "fricp_internal.cuh"
#include "select.cuh"
#include "solver.cuh"

namespace fricp {

namespace {

template <int K>
__device__ __forceinline__ void block_reduce_store(double (&acc)[K], double *out) {
    __shared__ double sm[kBlock / 32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sm[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) v += sm[w][threadIdx.x];
        out[threadIdx.x] = v;
    }
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

template <int VAR>
__global__ void __launch_bounds__(kBlock) k_step(StepArgs a) {
    constexpr int K = VAR ? kSumsP2PL : kSumsP2P;
    PairState *st = a.st;
    __shared__ double sR[9], sT[3], sC[3], sS[K];
    __shared__ double s_scale, s_inv2nu2;
    __shared__ float s_cut2;
    __shared__ int s_phase, s_done, s_welsch, s_M, s_last;
    if (threadIdx.x == 0) {
        s_done = st->done;
        s_phase = st->phase;
        s_welsch = st->variant != FRICP_P2P_AA;
        s_M = st->M;
        for (int i = 0; i < 9; ++i) sR[i] = st->Re[i];
        for (int r = 0; r < 3; ++r) {
            sT[r] = st->te[r];
            sC[r] = st->c[r];
        }
        s_scale = st->s;
        s_inv2nu2 = st->nu > 0.0 ? 1.0 / (2.0 * st->nu * st->nu) : 0.0;
        // cap radius in caller units: (d_n / s)^2 with d_n^2 / (2 nu^2) = kWelschCut
        const double cut2 = st->nu > 0.0 ? kWelschCut * 2.0 * st->nu * st->nu / (st->s * st->s) : 0.0;
        s_cut2 = (cut2 > 0.0 && cut2 < 3.0e38) ? (float)(cut2 * (1.0 + 1e-5)) : __int_as_float(0x7f800000);
    }
    __syncthreads();
    if (s_done) return;

    const int i = blockIdx.x * kBlock + threadIdx.x;
    const bool active = i < s_M;
    float4 p = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    double x[3] = {0.0, 0.0, 0.0};
    NNLane nq;
    if (active) {
        p = __ldg(a.src + i);
#pragma unroll
        for (int r = 0; r < 3; ++r)
            x[r] = fma(sR[3 * r], (double)p.x, fma(sR[3 * r + 1], (double)p.y, fma(sR[3 * r + 2], (double)p.z, sT[r])));
        nn_init(nq, x);
        const int j0 = a.prev[i];
        if (j0 >= 0) {   // warm start from the previous pass's correspondence
            const float4 q0 = __ldg(a.ix.pts + j0);
            nq.bestf = cand_d2f(nq, q0);
            nq.best64 = cand_d2_64(nq, q0);
            nq.best_j = j0;
            nq.best_orig = __float_as_int(q0.w);
        }
        // Welsch point-to-point: a point farther than the cap has weight
        // exp(-a) = 0.0 and psi = 1.0 exactly for every candidate that far, so
        // the search radius is capped there (the sums are bit-identical).
        if (VAR == 0 && s_welsch && s_phase != PH_INIT && s_cut2 < nq.bestf) nq.bestf = s_cut2;
        nn_thread(a.ix, nq);
        if (nq.best_j < 0) {   // nothing within the cap: any target point is equivalent
            nq.best_j = 0;
        }
    }

    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    if (active) {
        const int j = nq.best_j;
        a.prev[i] = j;
        const float4 q = __ldg(a.ix.pts + j);
        const double dx = x[0] - (double)q.x, dy = x[1] - (double)q.y, dz = x[2] - (double)q.z;
        const double s = s_scale;
        const double pt[3] = {(double)p.x - sC[0], (double)p.y - sC[1], (double)p.z - sC[2]};
        if (VAR == 0) {
            const double d2n = s * s * (dx * dx + dy * dy + dz * dz);
            double w, psi;
            if (s_welsch) {
                w = exp(-d2n * s_inv2nu2);
                psi = 1.0 - w;
            } else {
                w = 1.0;
                psi = d2n;
            }
            if (s_phase == PH_INIT) a.resid[i] = sqrt(d2n);
            const double qt[3] = {(double)q.x - sC[0], (double)q.y - sC[1], (double)q.z - sC[2]};
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
            const double h = s * (dx * n0 + dy * n1 + dz * n2);
            if (s_phase == PH_INIT) a.resid[i] = fabs(h);
            const double g = exp(-h * h * s_inv2nu2);
            // y = R p~ in normalised units; z = [y x n; n]
            double y[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) y[r] = s * (sR[3 * r] * pt[0] + sR[3 * r + 1] * pt[1] + sR[3 * r + 2] * pt[2]);
            const double z[6] = {y[1] * n2 - y[2] * n1, y[2] * n0 - y[0] * n2, y[0] * n1 - y[1] * n0, n0, n1, n2};
            int t = 0;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const double gz = g * z[r];
#pragma unroll
                for (int c = r; c < 6; ++c) acc[t++] = gz * z[c];
                acc[21 + r] = gz * h;
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
    if (s_phase == PH_INIT) {
        const int n = s_M;
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
    double x[3] = {0.0, 0.0, 0.0};
    NNLane q;
    if (active) {
        const double p0 = p[3 * i], p1 = p[3 * i + 1], p2 = p[3 * i + 2];
        for (int r = 0; r < 3; ++r) x[r] = fma(T[3 * r], p0, fma(T[3 * r + 1], p1, fma(T[3 * r + 2], p2, T[9 + r])));
        nn_init(q, x);
        nn_thread(ix, q);
        if (q.best_j < 0) q.best_j = 0;   // only for a non-finite x
    }
    if (active) {
        idx[i] = __float_as_int(__ldg(ix.pts + q.best_j).w);
        d2[i] = q.best64;
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

cudaError_t launch_step(const StepArgs &a, int variant, int ntiles, cudaStream_t s) {
    if (variant == FRICP_P2PL_WELSCH_AA)
        k_step<1><<<ntiles, kBlock, 0, s>>>(a);
    else
        k_step<0><<<ntiles, kBlock, 0, s>>>(a);
    counters().launches += 1;
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
        Index ix{t->pts, t->nrm, t->nodes, (int)t->n, t->L};
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
