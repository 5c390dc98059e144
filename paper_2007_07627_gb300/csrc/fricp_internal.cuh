// Internal declarations shared by the CUDA translation units of libfricp.
//
// Data layout in HBM (one target set Q, one registration):
//   pts   float4[n]      target points in Morton order; .w holds the original index bits
//   nrm   float4[n]      target normals in the same order (point-to-plane only)
//   nodes float4[4L]     complete binary box tree over L (power of two) buckets of
//                        kLeaf consecutive points; node i in [1, 2L) has its box at
//                        nodes[2i] (lo) and nodes[2i+1] (hi), so the two children of
//                        node i sit in one aligned 64-byte line nodes[4i .. 4i+3].
//                        Leaf l is node L + l; empty buckets have an inverted box.
//   src   float4[M]      source points in Morton order, .w = original index bits
//   PairState            one registration's solver state (FP64), ~2 KB
//   partial double[T][K] per-tile reduction records (T = ceil(M / kBlock) tiles)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fricp.h"

#define FRICP_HD __host__ __device__

namespace fricp {

constexpr int kBlock = 256;        // threads per step block = source points per tile
constexpr int kLeaf = 16;          // target points per bucket
constexpr int kStack = 32;         // traversal stack (tree depth <= 27 for n < 2^31)
constexpr int kMaxM = 5;           // largest Anderson history m
constexpr int kSumsP2P = 17;       // W, W p (3), W q (3), W p q^T (9), E
constexpr int kSumsP2PL = 28;      // g z z^T (21), g z B (6), E
constexpr int kMaxSums = 28;

// Relative slack of the box pruning test: a bucket is skipped only when its box
// distance exceeds the best distance by more than the float rounding of either.
constexpr float kShrink = 1.0f - 4e-6f;

// exp(-a) is 0.0 in FP64 for a > 745.14: a Welsch point-to-point residual with
// d^2 / (2 nu^2) >= kWelschCut has weight 0 and psi 1 exactly.
constexpr double kWelschCut = 750.0;

struct Index {
    const float4 *pts;
    const float4 *nrm;
    const float4 *nodes;
    int n;
    int L;
};

enum Phase : int {
    PH_INIT = 0,          // pass at T0 storing per-point residuals, then the nu_max median
    PH_STAGE_START = 1,   // pass at T^(k-1) with the new nu: first alignment of a stage
    PH_ITER = 2,          // pass at T^(k): energy check at the head of an inner iteration
    PH_ITER_REVERTED = 3, // pass at T' after a failed energy check (Alg. 1)
    PH_CAPCHECK = 4,      // pass at the iterate carried out of a stage on the cap
    PH_LS = 5,            // Alg. 2 line-search trial
    PH_EVAL = 6,          // single evaluation (fricp_eval_pass)
    PH_DONE = 7
};

struct PairState {
    // ---- problem (host-written before the first step)
    int variant;
    int m;
    int max_iters;
    int cap_first;
    int cap_max;
    int max_ls;
    int M;
    int ntiles;
    int trace_cap;
    int nu_max_given;
    double eps;
    double nu_max;
    double nu_min;
    double s;          // normalisation scale
    double c[3];       // normalisation centre (centroid of Q), caller units
    // ---- machine
    unsigned int counter;   // last-block ticket of the running step
    int phase;
    int done;
    int status;
    int n_body;             // inner bodies run in this stage: k - k_start - 1
    int cap;                // current I_nu
    int eval_counts;        // the pending pass is a new correspondence computation
    int capexit;            // the running line search started from a cap check
    int ls_l;
    int hlen;
    double nu;
    double E_prev;
    double tau;
    double E_best;
    // Alg. 1 transforms, normalised coordinates: R row-major (9) then t (3)
    double Tk[12], Tp[12], Tprev[12];
    double logTk[6], logTp[6];   // log of Tk / Tp, kept with them (one log per step)
    // Alg. 2 parameters xi = [delta; u]
    double xk[6], xprev[6], xstar[6], xeval[6], xbest[6];
    double sys_best[kMaxSums];
    // transform the next pass applies to the source, caller units: x = Re p + te
    double Re[9];
    double te[3];
    // Anderson history, oldest first: G^(k-j), F^(k-j)
    double Gh[kMaxM + 1][6];
    double Fh[kMaxM + 1][6];
    // counters
    int iterations, corr_passes, aa_accepted, reverts, ls_trials, stages, device_steps, trace_len;
    double final_energy;
    double eval_out[48];    // PH_EVAL result: E, T' or xi*, then the reduced sums
};

struct StepArgs {
    PairState *st;
    Index ix;
    const float4 *src;     // M sorted source points
    int *prev;             // M: correspondence (sorted target index) of the last pass, -1 if none
    double *partial;       // ntiles * kMaxSums
    double *resid;         // M per-point residuals (PH_INIT)
    double *trace;         // trace_cap energies
};

// ---------------------------------------------------------------------------
// Exact nearest neighbour (Sec. 3, Eq. 3) over the bucket tree, one query per
// thread (depth-first, nearer child first, pruned by the running bound).
//
// Precision: x is FP64. It is split once into xh = fl32(x), xl = fl32(x - xh);
// a candidate's difference (xh - q) + xl is formed in float, so its float
// squared distance has a relative error of a few float ulps (< 4e-7) however
// far x is from the origin. Every candidate whose float distance is within
// 2e-6 of the running float bound is re-ranked with its exact FP64 distance,
// and the winner is the lexicographic minimum of (FP64 d^2, original index): the
// FP64 argmin with ties to the lowest index. The bucket-pruning bound keeps a
// 4e-6 slack, so a bucket that may hold the FP64 winner is never skipped.
//
// Warm start: a query may start from any target point (the previous pass's
// correspondence); its distance is a true upper bound, so the result is the
// same exact argmin, found with far fewer node visits.
// ---------------------------------------------------------------------------
constexpr float kTieWindow = 1.0f + 2e-6f;

struct NNLane {
    double x[3];
    float xh[3], xl[3];
    float bestf;
    double best64;
    int best_j;
    int best_orig;
};

__device__ __forceinline__ void split_point(const double x[3], float xh[3], float xl[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xh[a] = __double2float_rn(x[a]);
        xl[a] = __double2float_rn(x[a] - (double)xh[a]);
    }
}

__device__ __forceinline__ float axis_gap(float lo, float hi, float xh, float xl) {
    return fmaxf(fmaxf((lo - xh) - xl, (xh - hi) + xl), 0.0f);
}

__device__ __forceinline__ float box_d2(float4 lo, float4 hi, const float xh[3], const float xl[3]) {
    const float a = axis_gap(lo.x, hi.x, xh[0], xl[0]);
    const float b = axis_gap(lo.y, hi.y, xh[1], xl[1]);
    const float c = axis_gap(lo.z, hi.z, xh[2], xl[2]);
    return fmaf(c, c, fmaf(b, b, a * a));
}

__device__ __forceinline__ float cand_d2f(const NNLane &q, float4 p) {
    const float dx = (q.xh[0] - p.x) + q.xl[0];
    const float dy = (q.xh[1] - p.y) + q.xl[1];
    const float dz = (q.xh[2] - p.z) + q.xl[2];
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

__device__ __forceinline__ double cand_d2_64(const NNLane &q, float4 p) {
    const double dx = q.x[0] - (double)p.x, dy = q.x[1] - (double)p.y, dz = q.x[2] - (double)p.z;
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ void nn_init(NNLane &q, const double x[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) q.x[a] = x[a];
    split_point(x, q.xh, q.xl);
    q.bestf = __int_as_float(0x7f800000);
    q.best64 = __longlong_as_double(0x7ff0000000000000ll);
    q.best_j = -1;
    q.best_orig = 0x7fffffff;
}

__device__ __forceinline__ void nn_offer(NNLane &q, float4 p, int j) {
    const float d = cand_d2f(q, p);
    if (d <= q.bestf * kTieWindow) {
        const double d64 = cand_d2_64(q, p);
        const int o = __float_as_int(p.w);
        if (d64 < q.best64 || (d64 == q.best64 && o < q.best_orig)) {
            q.best64 = d64;
            q.best_j = j;
            q.best_orig = o;
        }
        q.bestf = fminf(q.bestf, d);
    }
}

// Depth-first search from the root with the lane's current bound (q.bestf).
// A lane whose bound starts finite (warm start, or a radius cap) only visits
// buckets within that bound; if none holds a closer point the starting
// candidate stays (best_j may stay -1 when the search began from a bare cap).
__device__ __forceinline__ void nn_thread(const Index &ix, NNLane &q) {
    int stk[kStack];
    float stkd[kStack];
    int sp = 0;
    int node = 1;
    for (;;) {
        if (node < ix.L) {
            const float4 *b = ix.nodes + 4 * node;
            const float4 lo0 = __ldg(b), hi0 = __ldg(b + 1), lo1 = __ldg(b + 2), hi1 = __ldg(b + 3);
            float d0 = box_d2(lo0, hi0, q.xh, q.xl);
            float d1 = box_d2(lo1, hi1, q.xh, q.xl);
            int c0 = 2 * node, c1 = c0 + 1;
            if (d1 < d0) {
                const float td = d0; d0 = d1; d1 = td;
                const int tc = c0; c0 = c1; c1 = tc;
            }
            if (d0 * kShrink <= q.bestf) {
                if (d1 * kShrink <= q.bestf) {
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
            for (int j = beg; j < end; ++j) nn_offer(q, __ldg(ix.pts + j), j);
        }
        node = 0;
        while (sp > 0) {
            --sp;
            if (stkd[sp] * kShrink <= q.bestf) {
                node = stk[sp];
                break;
            }
        }
        if (node == 0) break;
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers (index.cu, step.cu). All return cudaError_t.
// ---------------------------------------------------------------------------
struct TargetDev {
    int64_t n;
    int L;
    int has_normals;
    float4 *pts;
    float4 *nrm;
    float4 *nodes;
    double centroid[3];
    float lo[3], hi[3];
    // nu_min statistics in caller units (median over q of the median 6-NN distance,
    // resp. plane distance); < 0 until computed.
    double E_Q, H_Q;
};

// Per-thread accounting behind fricp_counters (defined in api.cu).
struct Counters {
    int64_t launches, h2d, d2h;
};
Counters &counters();

// Defined in api.cu: the device view of a target handle, and the message that
// fricp_last_error returns on this thread.
const TargetDev *target_dev(const fricp_target *t);
void set_last_error(const char *msg);

cudaError_t build_target(const float *q_dev, const float *n_dev, int64_t n, cudaStream_t s,
                         TargetDev *t, int *bad_input);
cudaError_t target_nu_stats(TargetDev *t, cudaStream_t s);
cudaError_t prepare_source(const float *p_dev, int64_t m, cudaStream_t s, float4 *src_out,
                           float lo[3], float hi[3], int *bad_input);
cudaError_t launch_closest(const TargetDev *t, const float *p_dev, int64_t m, const double T[12],
                           int64_t *idx, double *d2, cudaStream_t s);
cudaError_t launch_step(const StepArgs &a, int variant, int ntiles, cudaStream_t s);
cudaError_t launch_setup_eval_xi(PairState *st, const double *T_normalized12, cudaStream_t s);

}  // namespace fricp
