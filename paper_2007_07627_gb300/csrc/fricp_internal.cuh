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
    double eval_out[16];    // PH_EVAL result
};

struct StepArgs {
    PairState *st;
    Index ix;
    const float4 *src;     // M sorted source points
    double *partial;       // ntiles * kMaxSums
    double *resid;         // M per-point residuals (PH_INIT)
    double *trace;         // trace_cap energies
};

// ---------------------------------------------------------------------------
// Exact nearest neighbour (Sec. 3, Eq. 3) over the bucket tree.
//
// x is the transformed source point in FP64. It is split once into
// xh = fl32(x), xl = fl32(x - xh); every candidate difference is formed as
// (xh - q) + xl in float, which carries x to about 2^-48 relative and rounds
// only relative to the difference itself, so the squared distance of every
// candidate has a relative error of a few float ulps even when x is far from
// the origin. Ties in the float distance go to the lowest original index.
// ---------------------------------------------------------------------------
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

__device__ __forceinline__ int nn_query(const Index &ix, const double x[3]) {
    float xh[3], xl[3];
    split_point(x, xh, xl);
    float best = __int_as_float(0x7f800000);  // +inf
    int best_j = -1;
    int best_orig = 0x7fffffff;
    int stk_node[kStack];
    float stk_d[kStack];
    int sp = 0;
    int node = 1;
    for (;;) {
        if (node < ix.L) {
            const float4 *b = ix.nodes + 4 * node;
            const float4 lo0 = __ldg(b), hi0 = __ldg(b + 1), lo1 = __ldg(b + 2), hi1 = __ldg(b + 3);
            float d0 = box_d2(lo0, hi0, xh, xl);
            float d1 = box_d2(lo1, hi1, xh, xl);
            int c0 = 2 * node, c1 = c0 + 1;
            if (d1 < d0) {
                const float td = d0; d0 = d1; d1 = td;
                const int tc = c0; c0 = c1; c1 = tc;
            }
            if (d0 * kShrink <= best) {
                if (d1 * kShrink <= best) {
                    stk_node[sp] = c1;
                    stk_d[sp] = d1;
                    ++sp;
                }
                node = c0;
                continue;
            }
        } else {
            const int beg = (node - ix.L) * kLeaf;
            const int end = min(beg + kLeaf, ix.n);
            for (int j = beg; j < end; ++j) {
                const float4 q = __ldg(ix.pts + j);
                const float dx = (xh[0] - q.x) + xl[0];
                const float dy = (xh[1] - q.y) + xl[1];
                const float dz = (xh[2] - q.z) + xl[2];
                const float d = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const int orig = __float_as_int(q.w);
                if (d < best || (d == best && orig < best_orig)) {
                    best = d;
                    best_j = j;
                    best_orig = orig;
                }
            }
        }
        node = 0;
        while (sp > 0) {
            --sp;
            if (stk_d[sp] * kShrink <= best) {
                node = stk_node[sp];
                break;
            }
        }
        if (node == 0) break;
    }
    // Only a non-finite x can leave nothing visited; index 0 keeps every read in bounds
    // and the non-finite distance flows into the sums.
    return best_j < 0 ? 0 : best_j;
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
