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
//   obb   float4[4L]     oriented box of every bucket (same allocation, after the
//                        nodes): centre c and half-extents h along three orthonormal
//                        axes a_k fitted to the bucket's points, as
//                        (c, h0) (a0, h1) (a1, h2) (a2, r), r the bucket's radius
//   src   float4[M]      source points in Morton order, .w = original index bits
//   PairState            one registration's solver state (FP64), ~2 KB
//   partial double[T][K] per-tile reduction records (T = ceil(M / kBlock) tiles)
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fricp.h"
#include "obb.cuh"

#define FRICP_HD __host__ __device__

namespace fricp {

constexpr int kBlock = 256;        // threads per step block = source points per tile
constexpr int kLeaf = 16;          // target points per bucket
constexpr int kStack = 64;         // traversal stack: path siblings + one descent <= 2 x depth (depth <= 27)
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

// Precision of a registration's search and per-point terms (fricp_params.precision):
//   PREC_FP64  candidates screened in float and re-ranked in double-float: the FP64
//              argmin, ties to the lowest original index; per-point terms in FP64;
//   PREC_FP32  transform, distances and weights in float (ties to the lowest
//              original index among equal float distances); sums and solve in FP64;
//   PREC_FP16  as PREC_FP32 on target coordinates stored as 16-bit offsets in their
//              bucket's box (8 B per point); ties to the lowest bucket-order position.
enum Prec : int { PREC_FP64 = 0, PREC_FP32 = 1, PREC_FP16 = 2 };

// Variant families: point-to-plane (the Alg. 2 scheme, 28 sums) and robust
// (Welsch weights and nu stages).
__host__ __device__ inline bool variant_p2pl(int v) {
    return v == FRICP_P2PL_WELSCH_AA || v == FRICP_P2PL_AA || v == FRICP_SYM_WELSCH_AA;
}
__host__ __device__ inline bool variant_robust(int v) {
    return v == FRICP_P2P_WELSCH_AA || v == FRICP_P2PL_WELSCH_AA || v == FRICP_SYM_WELSCH_AA;
}
// The symmetric objective: the point-to-plane scheme on a residual that also
// carries the source point's normal.
__host__ __device__ inline bool variant_sym(int v) { return v == FRICP_SYM_WELSCH_AA; }

struct Index {
    const float4 *pts;
    const float4 *nrm;
    const float4 *nodes;
    const ushort4 *pts16;   // FP16 storage (x, y, z as half offsets in the bucket box), or null
    int n;
    int L;
    const float4 *obb;      // oriented bucket boxes (4 float4 per bucket), or null: axis-aligned boxes only
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
    int prec;          // Prec
    double eps;
    double nu_max;
    double nu_min;
    double s;          // normalisation scale
    double c[3];       // normalisation centre (centroid of Q), caller units
    // ---- machine
    unsigned int counter;   // last-block ticket of the running step
    unsigned int nn_next;   // next work unit of the search kernel (query pair or query tile)
    int phase;
    int done;
    int status;
    int nn_overflow;        // a search kernel ran out of its bounded stack (sticky; reported as FRICP_EOVERFLOW)
    int n_body;             // inner bodies run in this stage: k - k_start - 1
    int cap;                // current I_nu
    int eval_counts;        // the pending pass is a new correspondence computation
    int capexit;            // the running line search started from a cap check
    int ls_l;
    int hlen;
    int init_median_ext;    // the first pass leaves the nu_max median to the host's grid-wide select (k_after_init)
    int pad0;
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
    // derived from Re, te and nu for the search and per-point kernels (set_head_cache):
    // float splits hi + lo of Re and te, 1 / (2 nu^2) and the Welsch cap radius^2 in caller units
    float hRh[9], hRl[9], hth[3], htl[3];
    float hcut2;
    double hinv2nu2;
    double hnu;   // nu that hinv2nu2 and hcut2 belong to (0: not set)
    // Anderson history, oldest first: G^(k-j), F^(k-j)
    double Gh[kMaxM + 1][6];
    double Fh[kMaxM + 1][6];
    // counters
    int iterations, corr_passes, aa_accepted, reverts, ls_trials, stages, device_steps, trace_len;
    double final_energy;
    double eval_out[48];    // PH_EVAL result: E, T' or xi*, then the reduced sums
    // normalised transform of the pass requested last (what a step record reports)
    double Teval[12];
    // per-pass records (fricp_register_recorded), or null
    fricp_step_record *rec;
    int rec_cap, rec_len;
};

struct StepArgs {
    PairState *st;
    Index ix;
    const float4 *src;     // M sorted source points
    const float4 *src_nrm = nullptr;   // M source normals in the same order (symmetric objective), or null
    int *prev;             // M: correspondence (sorted target index) of the last pass, -1 if none;
                           //    the search kernels overwrite it with this pass's correspondence
    double *partial;       // ntiles * kMaxSums
    double *resid;         // M per-point residuals (PH_INIT)
    double *trace;         // trace_cap energies
};

// ---------------------------------------------------------------------------
// Exact nearest neighbour (Sec. 3, Eq. 3) over the bucket tree, one query per
// thread (depth-first, nearer child first, pruned by the running bound).
//
// Precision: the search never touches the FP64 pipe (a few FP64 units per SM
// on this GPU). x = R p + t is formed in double-float arithmetic (a float pair
// hi + lo, error-free products and sums, about 2^-44 relative), so xh = hi and
// xl = lo carry x far beyond float precision. A candidate's float squared
// distance uses (xh - q) + xl, rounding only relative to the difference itself
// (relative error < 4e-7 however far x is from the origin). Every candidate
// whose float distance is within 2e-6 of the running float bound is re-ranked
// by its double-float squared distance, and the winner is the lexicographic
// minimum of (that distance, original index): the exact argmin up to ties
// closer than about 1e-10 relative, ties to the lowest index. The
// bucket-pruning bound keeps a 4e-6 slack, so a bucket that may hold the
// winner is never skipped.
//
// Warm start: a query may start from any target point (the previous pass's
// correspondence); its distance is a true upper bound, so the result is the
// same argmin, found with far fewer node visits.
// ---------------------------------------------------------------------------
constexpr float kTieWindow = 1.0f + 2e-6f;

struct NNLane {
    float xh[3], xl[3];
    float xdn[3], xup[3];    // xh + xl rounded down and up: float bounds of x for the box tests
    float bestf;             // float bound (smallest float distance seen)
    float best_hi, best_lo;  // double-float squared distance of the winner
    int best_j;
    int best_orig;
};

// Error-free transformations (Knuth two-sum, FMA two-product) and a
// double-float sum renormalised so that |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl) {
    float s, e;
    two_sum(h, bh, s, e);
    e += l + bl;
    h = s + e;
    l = e - (h - s);
}

// x = R p + t in double-float from float splits of the FP64 R and t.
__device__ __forceinline__ void df_transform(const float Rh[9], const float Rl[9], const float th[3],
                                             const float tl[3], float4 p, float xh[3], float xl[3]) {
    const float pv[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float h = th[a], l = tl[a];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float ph = Rh[3 * a + j] * pv[j];
            float pe = fmaf(Rh[3 * a + j], pv[j], -ph);
            pe = fmaf(Rl[3 * a + j], pv[j], pe);
            df_add(h, l, ph, pe);
        }
        xh[a] = h;
        xl[a] = l;
    }
}

// Split an FP64 value into a float pair (host or device set-up code).
FRICP_HD inline void split_double(double v, float &h, float &l) {
    h = (float)v;
    l = (float)(v - (double)h);
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

// Squared distance from x = xh + xl to a bucket's oriented box (obb_fit,
// obb_eval in obb.cuh): at most (1 + 8e-6) times the squared distance to the
// bucket's nearest point. A bucket is skipped only when this distance, shrunk by
// kObbShrink, still exceeds the bound: it can never hold a point inside the tie
// window.
constexpr float kObbShrink = 1.0f - 2e-5f;

__device__ __forceinline__ float obb_d2(const float4 *o, const float xh[3], const float xl[3]) {
    return obb_eval(__ldg(o), __ldg(o + 1), __ldg(o + 2), __ldg(o + 3), xh, xl);
}

// Box test of a search lane: xdn <= x <= xup on every axis, so lo - xup and
// xdn - hi never exceed the true gaps lo - x and x - hi (each subtraction then
// rounds relative to its result, which kShrink covers): two operations per axis
// fewer than box_d2 on the double-float pair.
__device__ __forceinline__ float box_d2q(float4 lo, float4 hi, const NNLane &q) {
    const float a = fmaxf(fmaxf(lo.x - q.xup[0], q.xdn[0] - hi.x), 0.0f);
    const float b = fmaxf(fmaxf(lo.y - q.xup[1], q.xdn[1] - hi.y), 0.0f);
    const float c = fmaxf(fmaxf(lo.z - q.xup[2], q.xdn[2] - hi.z), 0.0f);
    return fmaf(c, c, fmaf(b, b, a * a));
}

__device__ __forceinline__ float cand_d2f(const NNLane &q, float4 p) {
    const float dx = (q.xh[0] - p.x) + q.xl[0];
    const float dy = (q.xh[1] - p.y) + q.xl[1];
    const float dz = (q.xh[2] - p.z) + q.xl[2];
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// Squared distance in double-float: (xh - q) is split exactly by two-sum, xl
// added, each difference squared by two-product.
__device__ __forceinline__ void cand_d2_df(const NNLane &q, float4 p, float &hi, float &lo) {
    const float pv[3] = {p.x, p.y, p.z};
    hi = 0.0f;
    lo = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float s, e;
        two_sum(q.xh[a], -pv[a], s, e);
        e += q.xl[a];
        const float dh = s + e;
        const float dl = e - (dh - s);
        const float sq = dh * dh;
        float sqe = fmaf(dh, dh, -sq);
        sqe = fmaf(2.0f * dh, dl, sqe);
        df_add(hi, lo, sq, sqe);
    }
}

__device__ __forceinline__ void nn_init(NNLane &q, const float xh[3], const float xl[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q.xh[a] = xh[a];
        q.xl[a] = xl[a];
        q.xdn[a] = __fadd_rd(xh[a], xl[a]);
        q.xup[a] = __fadd_ru(xh[a], xl[a]);
    }
    q.bestf = __int_as_float(0x7f800000);
    q.best_hi = __int_as_float(0x7f800000);
    q.best_lo = 0.0f;
    q.best_j = -1;
    q.best_orig = 0x7fffffff;
}

// Make candidate p (sorted index j) the current winner unconditionally (warm start).
template <int PREC = PREC_FP64>
__device__ __forceinline__ void nn_seed(NNLane &q, float4 p, int j) {
    q.bestf = cand_d2f(q, p);
    if (PREC == PREC_FP64) {
        cand_d2_df(q, p, q.best_hi, q.best_lo);
    } else {
        q.best_hi = q.bestf;
        q.best_lo = 0.0f;
    }
    q.best_j = j;
    q.best_orig = __float_as_int(p.w);
}

// Target point j as the search and the per-point terms see it at precision PREC
// (.w: the tie-break key: original index, or the bucket-order position for FP16).
template <int PREC>
__device__ __forceinline__ float4 target_point(const Index &ix, int j) {
    if (PREC != PREC_FP16) return __ldg(ix.pts + j);
    const ushort4 h = __ldg(ix.pts16 + j);
    const int leaf = ix.L + j / kLeaf;
    const float4 lo = __ldg(ix.nodes + 2 * leaf), hi = __ldg(ix.nodes + 2 * leaf + 1);
    float4 r;
    r.x = fmaf(__half2float(__ushort_as_half(h.x)), hi.x - lo.x, lo.x);
    r.y = fmaf(__half2float(__ushort_as_half(h.y)), hi.y - lo.y, lo.y);
    r.z = fmaf(__half2float(__ushort_as_half(h.z)), hi.z - lo.z, lo.z);
    r.w = __int_as_float(j);
    return r;
}

// (double-float d^2, original index) lexicographic order; both pairs are
// renormalised, so (hi, lo) order is the order of hi + lo.
__device__ __forceinline__ bool lex_less(float ha, float la, int oa, float hb, float lb, int ob) {
    return ha < hb || (ha == hb && (la < lb || (la == lb && oa < ob)));
}

// Returns true when p entered the tie window (the lane's bound or winner may change).
template <int PREC = PREC_FP64>
__device__ __forceinline__ bool nn_offer(NNLane &q, float4 p, int j) {
    const float d = cand_d2f(q, p);
    if (d <= q.bestf * kTieWindow) {
        float hi = d, lo = 0.0f;
        if (PREC == PREC_FP64) cand_d2_df(q, p, hi, lo);
        const int o = __float_as_int(p.w);
        if (lex_less(hi, lo, o, q.best_hi, q.best_lo, q.best_orig)) {
            q.best_hi = hi;
            q.best_lo = lo;
            q.best_j = j;
            q.best_orig = o;
        }
        q.bestf = fminf(q.bestf, d);
        return true;
    }
    return false;
}

// Whether leaf node `leaf` (L + bucket) may hold a point within the lane's
// bound by its oriented box (its axis-aligned box passed already). FP16
// storage decodes points inside the axis-aligned box only, so it skips this test.
template <int PREC = PREC_FP64>
__device__ __forceinline__ bool obb_meets(const Index &ix, const NNLane &q, int leaf) {
    if (PREC == PREC_FP16 || ix.obb == nullptr) return true;
    return obb_d2(ix.obb + 4 * (leaf - ix.L), q.xh, q.xl) * kObbShrink <= q.bestf;
}

// Depth-first search from the root with the lane's current bound (q.bestf).
// A lane whose bound starts finite (warm start, or a radius cap) only visits
// buckets within that bound; if none holds a closer point the starting
// candidate stays (best_j may stay -1 when the search began from a bare cap).
// start_leaf >= 0 (the bucket of a warm-start candidate): the search begins at
// that bucket instead of the root. The siblings of the bucket's path to the
// root are pushed first (their subtrees partition the rest of the tree), the
// deepest on top, each with its box distance; the bucket itself is scanned
// first. Near the previous correspondence the bound then prunes almost every
// sibling at once, so a search costs a few memory latencies instead of one per
// tree level. The set of points examined is still every point that can beat
// the bound, so the result is the same exact argmin.
__device__ __forceinline__ void nn_thread(const Index &ix, NNLane &q, int start_leaf = -1) {
    int stk[kStack];
    float stkd[kStack];
    int sp = 0;
    int node = 1;
    if (start_leaf >= 0) {
        int sib[kStack];
        int ns = 0;
        for (int a = ix.L + start_leaf; a > 1; a >>= 1) sib[ns++] = a ^ 1;
        for (int k = ns - 1; k >= 0; --k) {
            const int c = sib[k];
            const float d = box_d2q(__ldg(ix.nodes + 2 * c), __ldg(ix.nodes + 2 * c + 1), q);
            if (d * kShrink <= q.bestf) {
                stk[sp] = c;
                stkd[sp] = d;
                ++sp;
            }
        }
        node = ix.L + start_leaf;
    }
    for (;;) {
        if (node < ix.L) {
            const float4 *b = ix.nodes + 4 * node;
            const float4 lo0 = __ldg(b), hi0 = __ldg(b + 1), lo1 = __ldg(b + 2), hi1 = __ldg(b + 3);
            float d0 = box_d2q(lo0, hi0, q);
            float d1 = box_d2q(lo1, hi1, q);
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
        } else if (obb_meets(ix, q, node)) {
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
// One query searched by a whole warp (all lanes hold the same query). The
// search starts at a bucket: the warm-start candidate's, or for a cold query
// the bucket reached by descending to the nearer child at every level. The
// siblings of that bucket's path to the root are tested in parallel (one per
// lane) and pushed on a warp-shared stack, deepest on top, with the bucket
// itself on top of them. Each round the lanes pop up to 32 nodes:
//   - an internal node pushes its children that pass the bound (two ballots
//     compact the pushes: farther children below nearer ones);
//   - the points of the popped buckets are spread over the lanes, two buckets
//     per pass of 16 lanes each;
// and the float bound is then reduced across the warp so every lane prunes
// with the same bound; the lexicographic (FP64 d^2, original index) minimum of
// the lanes' winners is reduced once, at the end. Every point that can beat
// the bound is examined, so the result is the same exact argmin as a serial
// depth-first search.
// ---------------------------------------------------------------------------
constexpr int kWarpStack = 1024;  // per warp; a round grows the stack by <= 96

// The float bound alone, min over the warp: what the pruning of the next round
// needs. Each lane keeps the lexicographic winner of the candidates it was
// offered; their minimum (warp_best) is taken once, when the search ends. The
// candidates a lane accepts depend only on the bound, so the winner is the same
// as with a full reduction every round.
__device__ __forceinline__ void warp_min_bound(NNLane &q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q.bestf = fminf(q.bestf, __shfl_xor_sync(0xffffffffu, q.bestf, o));
}

__device__ __forceinline__ void warp_best(NNLane &q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, q.best_hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, q.best_lo, o);
        const int oo = __shfl_xor_sync(0xffffffffu, q.best_orig, o);
        const int oj = __shfl_xor_sync(0xffffffffu, q.best_j, o);
        const float of = __shfl_xor_sync(0xffffffffu, q.bestf, o);
        if (lex_less(oh, ol, oo, q.best_hi, q.best_lo, q.best_orig)) {
            q.best_hi = oh;
            q.best_lo = ol;
            q.best_orig = oo;
            q.best_j = oj;
        }
        q.bestf = fminf(q.bestf, of);
    }
}

// Returns false if the stack would overflow (the caller flags it as an error).
template <int PREC>
__device__ __forceinline__ bool warp_nn(const Index &ix, NNLane &q, int *stk, int start_leaf) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    int depth = 0;
    while ((1 << depth) < ix.L) ++depth;
    if (start_leaf < 0) {   // cold: greedy descent (uniform: every lane computes the same)
        int node = 1;
        while (node < ix.L) {
            const float4 *b = ix.nodes + 4 * node;
            const float d0 = box_d2q(__ldg(b), __ldg(b + 1), q);
            const float d1 = box_d2q(__ldg(b + 2), __ldg(b + 3), q);
            node = 2 * node + (d1 < d0 ? 1 : 0);
        }
        start_leaf = node - ix.L;
    }
    int sp;
    {
        int c = 0;
        bool pass = false;
        if (lane < depth) {   // the sibling of the path node at level lane + 1
            c = ((ix.L + start_leaf) >> (depth - 1 - lane)) ^ 1;
            pass = box_d2q(__ldg(ix.nodes + 2 * c), __ldg(ix.nodes + 2 * c + 1), q) * kShrink <= q.bestf;
        }
        const unsigned m = __ballot_sync(FULL, pass);
        if (pass) stk[__popc(m & below)] = c;
        sp = __popc(m);
        if (lane == 0) stk[sp] = ix.L + start_leaf;
        ++sp;
    }
    __syncwarp();
    const int leaf_parent_level = depth - 1;   // nodes at this level have bucket children
    while (sp > 0) {
        const int k = min(32, sp);
        const int node = (lane < k) ? stk[sp - 1 - lane] : 0;
        sp -= k;
        __syncwarp();
        // An internal node two or more levels above the buckets is expanded to
        // its four grandchildren (boxes in two adjacent 64-byte lines), a node
        // just above the buckets to its two children: two levels per round.
        int c[4] = {0, 0, 0, 0};
        bool ok[4] = {false, false, false, false};
        bool leaf_ok = false;
        if (node != 0) {
            if (node < ix.L) {
                const int level = 31 - __clz(node);
                if (level < leaf_parent_level) {
                    const float4 *b = ix.nodes + 8 * node;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        c[g] = 4 * node + g;
                        ok[g] = box_d2q(__ldg(b + 2 * g), __ldg(b + 2 * g + 1), q) * kShrink <= q.bestf;
                    }
                } else {
                    const float4 *b = ix.nodes + 4 * node;
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        c[g] = 2 * node + g;
                        ok[g] = box_d2q(__ldg(b + 2 * g), __ldg(b + 2 * g + 1), q) * kShrink <= q.bestf;
                    }
                }
            } else {
                leaf_ok = box_d2q(__ldg(ix.nodes + 2 * node), __ldg(ix.nodes + 2 * node + 1), q) * kShrink
                              <= q.bestf &&
                          obb_meets<PREC>(ix, q, node);
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
        bool changed = false;
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
            if (lane < 16 || two) {
                const int j = ((lane < 16 ? na : nb) - ix.L) * kLeaf + (lane & 15);
                if (j < ix.n) changed |= nn_offer<PREC>(q, target_point<PREC>(ix, j), j);
            }
        }
        if (__ballot_sync(FULL, changed)) warp_min_bound(q);   // only when some lane's bound moved
        __syncwarp();
    }
    warp_best(q);
    return true;
}

// ---------------------------------------------------------------------------
// Half-warp form of warp_nn: lanes 0-15 search one query and lanes 16-31
// another, each half with its own lane state, its own stack (kHalfStack
// entries) and its own rounds. A warm-started query pops about nine nodes per
// round, so one query per warp leaves most lanes idle in the box tests; two
// queries share the instruction stream instead. Every warp-wide primitive is
// run by all 32 lanes and each half reads its own 16 bits; a half without a
// query (`live` false) only takes part in them. Returns false (for both
// halves) if either stack would overflow.
// ---------------------------------------------------------------------------
constexpr int kHalfStack = kWarpStack / 2;

__device__ __forceinline__ void half_min_bound(NNLane &q) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) q.bestf = fminf(q.bestf, __shfl_xor_sync(0xffffffffu, q.bestf, o));
}

__device__ __forceinline__ void half_best(NNLane &q) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {   // xor below 16 stays inside the half
        const float oh = __shfl_xor_sync(0xffffffffu, q.best_hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, q.best_lo, o);
        const int oo = __shfl_xor_sync(0xffffffffu, q.best_orig, o);
        const int oj = __shfl_xor_sync(0xffffffffu, q.best_j, o);
        const float of = __shfl_xor_sync(0xffffffffu, q.bestf, o);
        if (lex_less(oh, ol, oo, q.best_hi, q.best_lo, q.best_orig)) {
            q.best_hi = oh;
            q.best_lo = ol;
            q.best_orig = oo;
            q.best_j = oj;
        }
        q.bestf = fminf(q.bestf, of);
    }
}

template <int PREC>
__device__ __forceinline__ bool halfwarp_nn(const Index &ix, NNLane &q, int *stk, int start_leaf, bool live) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int hl = lane & 15;
    const int hs = lane & 16;
    const unsigned hmask = 0xffffu << hs;
    const unsigned below = ((1u << hl) - 1u) << hs;
    int depth = 0;
    while ((1 << depth) < ix.L) ++depth;
    if (live && start_leaf < 0) {   // cold: greedy descent (uniform within the half)
        int node = 1;
        while (node < ix.L) {
            const float4 *b = ix.nodes + 4 * node;
            const float d0 = box_d2q(__ldg(b), __ldg(b + 1), q);
            const float d1 = box_d2q(__ldg(b + 2), __ldg(b + 3), q);
            node = 2 * node + (d1 < d0 ? 1 : 0);
        }
        start_leaf = node - ix.L;
    }
    int sp = 0;
    for (int lv0 = 0; lv0 < depth; lv0 += 16) {   // siblings of the path, root side first
        const int lv = lv0 + hl;
        int c = 0;
        bool pass = false;
        if (live && lv < depth) {
            c = ((ix.L + start_leaf) >> (depth - 1 - lv)) ^ 1;
            pass = box_d2q(__ldg(ix.nodes + 2 * c), __ldg(ix.nodes + 2 * c + 1), q) * kShrink <= q.bestf;
        }
        const unsigned m = __ballot_sync(FULL, pass) & hmask;
        if (pass) stk[sp + __popc(m & below)] = c;
        sp += __popc(m);
    }
    if (live) {
        if (hl == 0) stk[sp] = ix.L + start_leaf;
        ++sp;
    }
    __syncwarp();
    const int leaf_parent_level = depth - 1;
    bool ovf = false;
    while (__any_sync(FULL, sp > 0)) {
        const int k = min(16, sp);
        const int node = (hl < k) ? stk[sp - 1 - hl] : 0;
        sp -= k;
        __syncwarp();
        int c[4] = {0, 0, 0, 0};
        bool ok[4] = {false, false, false, false};
        bool leaf_ok = false;
        if (node != 0) {
            if (node < ix.L) {
                const int level = 31 - __clz(node);
                if (level < leaf_parent_level) {
                    const float4 *b = ix.nodes + 8 * node;
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        c[g] = 4 * node + g;
                        ok[g] = box_d2q(__ldg(b + 2 * g), __ldg(b + 2 * g + 1), q) * kShrink <= q.bestf;
                    }
                } else {
                    const float4 *b = ix.nodes + 4 * node;
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        c[g] = 2 * node + g;
                        ok[g] = box_d2q(__ldg(b + 2 * g), __ldg(b + 2 * g + 1), q) * kShrink <= q.bestf;
                    }
                }
            } else {
                leaf_ok = box_d2q(__ldg(ix.nodes + 2 * node), __ldg(ix.nodes + 2 * node + 1), q) * kShrink
                              <= q.bestf &&
                          obb_meets<PREC>(ix, q, node);
            }
        }
        int base = sp;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const unsigned mg = __ballot_sync(FULL, ok[g]) & hmask;
            if (base + __popc(mg) > kHalfStack) ovf = true;
            else if (ok[g]) stk[base + __popc(mg & below)] = c[g];
            if (!ovf) base += __popc(mg);
        }
        sp = base;
        if (__any_sync(FULL, ovf)) return false;
        unsigned lm = __ballot_sync(FULL, leaf_ok) & hmask;
        bool changed = false;
        while (__any_sync(FULL, lm != 0u)) {   // one bucket per half per pass
            const bool have = lm != 0u;
            int src = lane;
            if (have) {
                src = __ffs(lm) - 1;
                lm &= lm - 1u;
            }
            const int na = __shfl_sync(FULL, node, src);
            if (have) {
                const int j = (na - ix.L) * kLeaf + hl;
                if (j < ix.n) changed |= nn_offer<PREC>(q, target_point<PREC>(ix, j), j);
            }
        }
        if (__any_sync(FULL, changed)) half_min_bound(q);
        __syncwarp();
    }
    half_best(q);
    return true;
}

// ---------------------------------------------------------------------------
// Query tile: a warp holds kTileQ = 8 Morton-adjacent queries, each on a
// group of four lanes (lane = 4 g + u: query g, sub-lane u; the four lanes of
// a group carry the same query and the same warm start: the bound is the
// distance to the previous pass's correspondence, or the Welsch cap).
// Adjacent queries need mostly the same part of the tree, so the warp walks
// it once for all eight:
//   - from the bucket of one query's warm start, the siblings of that
//     bucket's path to the root are tested (their subtrees partition the rest
//     of the tree), then the children of every node kept, up to 32 nodes a
//     round: sub-lane u tests the children of nodes u, u + 4, ... of the round
//     against its own query's ball with the pruning test of the serial search,
//     and a node is kept when it is within some query's bound;
//   - the buckets kept are staged, two per pass, in shared memory (one
//     coalesced 16-byte load per lane; FP16 storage is decoded here, once per
//     point); sub-lane u offers staged points u, u + 4, ..., u + 28 to its
//     query, and the group shares its float bound after every pass.
// When the walk ends, the four sub-lanes' winners are reduced to the
// lexicographic (FP64 distance, index) minimum. Every point that can beat a
// query's bound lies in a bucket whose ancestors and itself passed that
// query's test, and whichever sub-lane is offered the argmin keeps it (its
// float distance is within the tie window of any bound), so the result is the
// exact argmin of the serial search, ties included. A query far from the
// others costs its own ball's nodes, not a box around everybody's.
//
// Queries without a warm start (the first pass) are set aside, and so is
// every query of a tile whose walk would overflow its stack or bucket list
// (not expected): the caller searches them one by one with the whole warp
// (warp_nn). Returns the ballot mask of the lanes whose query is set aside (all
// four lanes of a group); their state is undefined.
//
// Per warp: `stk` kTileStack ints and `pend` kTilePend ints (which warp_nn may
// reuse as its stack afterwards: kTileStack + kTilePend <= kWarpStack), and
// `stage` kRing x 32 float4.
// ---------------------------------------------------------------------------
constexpr int kTileQ = 8;             // queries per warp
constexpr int kTileStack = 512;       // nodes kept and not yet expanded
constexpr int kTileDrain = 16;        // buckets kept before they are scanned
constexpr int kTilePend = kTileDrain + 64;   // a round adds <= 64, the path siblings <= 27
static_assert(kTileStack + kTilePend <= kWarpStack, "tile buffers share the per-warp search stack");

// Lexicographic winner and float bound of the four lanes of a group.
__device__ __forceinline__ void group4_best(NNLane &q) {
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, q.best_hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, q.best_lo, o);
        const int oo = __shfl_xor_sync(0xffffffffu, q.best_orig, o);
        const int oj = __shfl_xor_sync(0xffffffffu, q.best_j, o);
        const float of = __shfl_xor_sync(0xffffffffu, q.bestf, o);
        if (lex_less(oh, ol, oo, q.best_hi, q.best_lo, q.best_orig)) {
            q.best_hi = oh;
            q.best_lo = ol;
            q.best_orig = oo;
            q.best_j = oj;
        }
        q.bestf = fminf(q.bestf, of);
    }
}

__device__ __forceinline__ bool ball_meets(const NNLane &q, bool easy, float4 lo, float4 hi) {
    return easy && box_d2q(lo, hi, q) * kShrink <= q.bestf;
}

// Asynchronous 16-byte global -> shared copies (cp.async, cached in L1).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int kRing = 4;   // bucket pairs in flight in the scan (stage: kRing x 32 float4 per warp)

// Scan the buckets pend[0 .. np), two per pass. FP32/FP64 storage: the pairs
// stream through a ring of kRing stage slots with asynchronous copies, so
// kRing - 1 pairs are in flight while one is offered; FP16 storage is decoded
// by each lane on the way in.
template <int PREC>
__device__ __forceinline__ void tile_scan(const Index &ix, NNLane &q, bool easy, const int *pend, int np,
                                          float4 *stage) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int u = lane & 3;
    const float INF = __int_as_float(0x7f800000);
    const int npairs = (np + 1) >> 1;
    // pair k -> ring slot k % kRing: lane l brings point l & 15 of bucket 2k (l < 16) or 2k + 1
    auto issue = [&](int k) {
        if (k < npairs) {
            const int mine = (lane < 16) ? pend[2 * k] : (2 * k + 1 < np ? pend[2 * k + 1] : -1);
            const int jm = (mine - ix.L) * kLeaf + (lane & 15);
            float4 *dst = stage + (k % kRing) * 32 + lane;
            if (mine >= 0 && jm < ix.n) {
                if (PREC == PREC_FP16)
                    *dst = target_point<PREC>(ix, jm);
                else
                    cp_async16(dst, ix.pts + jm);
            } else {
                *dst = make_float4(INF, INF, INF, 0.0f);
            }
        }
        cp_async_commit();   // one group per call, empty or not, so the counting below holds
    };
#pragma unroll
    for (int k = 0; k < kRing - 1; ++k) issue(k);
    for (int k = 0; k < npairs; ++k) {
        issue(k + kRing - 1);          // into the slot consumed in the previous round
        cp_async_wait<kRing - 1>();    // this lane's copy of pair k has landed
        __syncwarp();                  // ... and every lane's
        const float4 *sl = stage + (k % kRing) * 32;
        if (easy) {
            const int la = pend[2 * k];
            const int lb = (2 * k + 1 < np) ? pend[2 * k + 1] : la;
            const int ja = (la - ix.L) * kLeaf, jb = (lb - ix.L) * kLeaf;
#pragma unroll
            for (int t = 0; t < 4; ++t) nn_offer<PREC>(q, sl[4 * t + u], ja + 4 * t + u);
#pragma unroll
            for (int t = 0; t < 4; ++t) nn_offer<PREC>(q, sl[16 + 4 * t + u], jb + 4 * t + u);
        }
        // the group shares its float bound (the winners are reduced at the end)
        q.bestf = fminf(q.bestf, __shfl_xor_sync(FULL, q.bestf, 1));
        q.bestf = fminf(q.bestf, __shfl_xor_sync(FULL, q.bestf, 2));
        __syncwarp();                  // slot k % kRing is free for pair k + kRing
    }
    cp_async_wait<0>();
    __syncwarp();
}

// Append the nodes of `cand` (lanes t < nc hold one each) whose bit is set in
// `keep`: buckets to pend, inner nodes to the stack. Returns false when either
// would overflow.
__device__ __forceinline__ bool tile_keep(const Index &ix, int cand, int nc, unsigned keep, int *stk, int &sp,
                                          int *pend, int &np) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const bool kept = lane < nc && ((keep >> lane) & 1u);
    const unsigned ml = __ballot_sync(FULL, kept && cand >= ix.L);
    const unsigned mi = __ballot_sync(FULL, kept && cand < ix.L);
    if (np + __popc(ml) > kTilePend || sp + __popc(mi) > kTileStack) return false;
    if (kept && cand >= ix.L) pend[np + __popc(ml & below)] = cand;
    if (kept && cand < ix.L) stk[sp + __popc(mi & below)] = cand;
    np += __popc(ml);
    sp += __popc(mi);
    __syncwarp();
    return true;
}

template <int PREC>
__device__ __forceinline__ unsigned tile_nn(const Index &ix, NNLane &q, bool live, int *stk, int *pend,
                                            float4 *stage) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int u = lane & 3;
    const float INF = __int_as_float(0x7f800000);
    const bool easy = live && q.best_j >= 0 && q.bestf < INF;
    const unsigned emask = __ballot_sync(FULL, easy);
    const unsigned cold = __ballot_sync(FULL, live && !easy);
    if (emask == 0u) return cold;
    int depth = 0;
    while ((1 << depth) < ix.L) ++depth;
    const int start = ix.L + __shfl_sync(FULL, q.best_j, __ffs(emask) - 1) / kLeaf;
    int sp = 0, np = 0;
    bool ok = true;
    // the start bucket holds a warm-start point: it is within that query's bound
    if (lane == 0) pend[0] = start;
    np = 1;
    // the siblings of the start bucket's path, root side first (so the deepest
    // ends on top of the stack), in batches of eight
    for (int k0 = 0; k0 < depth && ok; k0 += 8) {
        int nd[2];
        bool pass[2];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int k = k0 + 4 * v + u;
            nd[v] = k < depth ? (start >> (depth - 1 - k)) ^ 1 : 0;
            pass[v] = nd[v] != 0 && ball_meets(q, easy, __ldg(ix.nodes + 2 * nd[v]), __ldg(ix.nodes + 2 * nd[v] + 1));
        }
        const unsigned m0 = __ballot_sync(FULL, pass[0]), m1 = __ballot_sync(FULL, pass[1]);
        // lane t < 8 stands for sibling k0 + t (held by sub-lane t & 3 in slot t >> 2)
        const int o0 = __shfl_sync(FULL, nd[0], lane & 3), o1 = __shfl_sync(FULL, nd[1], lane & 3);
        const int cand = (lane >> 2) == 0 ? o0 : o1;
        const unsigned keep = ((m0 & 0x11111111u) ? 1u : 0u) | ((m0 & 0x22222222u) ? 2u : 0u) |
                              ((m0 & 0x44444444u) ? 4u : 0u) | ((m0 & 0x88888888u) ? 8u : 0u) |
                              ((m1 & 0x11111111u) ? 16u : 0u) | ((m1 & 0x22222222u) ? 32u : 0u) |
                              ((m1 & 0x44444444u) ? 64u : 0u) | ((m1 & 0x88888888u) ? 128u : 0u);
        ok = tile_keep(ix, cand, min(8, depth - k0), keep, stk, sp, pend, np);
    }
    while (ok && (sp > 0 || np > 0)) {
        if (np >= kTileDrain || (sp == 0 && np > 0)) {
            tile_scan<PREC>(ix, q, easy, pend, np, stage);
            np = 0;
        }
        if (sp == 0) break;
        // pop up to 32 nodes; sub-lane u expands nodes u, u + 4, ..., u + 28
        // (slot v holds node 4 v + u): a small walk uses the first slots only,
        // a large one expands 32 nodes per round
        const int k = min(32, sp);
        const int nslot = (k + 3) >> 2;
        int nd[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) nd[v] = (4 * v + u < k) ? stk[sp - 1 - (4 * v + u)] : 0;
        sp -= k;
        __syncwarp();
        unsigned keep[2] = {0u, 0u};   // bit 2 (4 v + u') + c of word v >> 2: child c of node 4 v + u'
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            if (v < nslot) {
                bool pass0 = false, pass1 = false;
                if (nd[v] != 0) {
                    const float4 *b = ix.nodes + 4 * nd[v];
                    pass0 = ball_meets(q, easy, __ldg(b), __ldg(b + 1));
                    pass1 = ball_meets(q, easy, __ldg(b + 2), __ldg(b + 3));
                }
                unsigned m0 = __ballot_sync(FULL, pass0), m1 = __ballot_sync(FULL, pass1);
                // fold the eight groups: bit w of the low nibble = some query kept it
                m0 |= m0 >> 16; m0 |= m0 >> 8; m0 |= m0 >> 4;
                m1 |= m1 >> 16; m1 |= m1 >> 8; m1 |= m1 >> 4;
                unsigned bits = 0u;
#pragma unroll
                for (int w = 0; w < 4; ++w) bits |= (((m0 >> w) & 1u) << (2 * w)) | (((m1 >> w) & 1u) << (2 * w + 1));
                keep[v >> 2] |= bits << (8 * (v & 3));
            }
        }
        // lane t stands for child t & 1 of node (t >> 1) + 16 h (h: the word),
        // held by sub-lane (t >> 1) & 3 in slot (t >> 3) + 4 h
        const int src = (lane >> 1) & 3;
#pragma unroll
        for (int hw = 0; hw < 2; ++hw) {
            if (16 * hw < k) {
                int cand = 0;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int o = __shfl_sync(FULL, nd[4 * hw + v], src);
                    if ((lane >> 3) == v) cand = 2 * o + (lane & 1);
                }
                ok = ok && tile_keep(ix, cand, min(32, 2 * (k - 16 * hw)), keep[hw], stk, sp, pend, np);
            }
        }
    }
    if (!ok) return __ballot_sync(FULL, live);
    group4_best(q);
    return cold;
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
    float4 *nodes;    // 4L float4 of boxes, then 4L float4 of oriented bucket boxes (one allocation)
    float4 *obb;      // = nodes + 4L
    ushort4 *pts16;   // FP16 storage, built on first use (build_fp16_storage)
    double centroid[3];
    float lo[3], hi[3];
    // nu_min statistics in caller units (median over q of the median 6-NN distance,
    // resp. plane distance); < 0 until computed.
    double E_Q, H_Q;
};

inline Index make_index(const TargetDev &t) { return Index{t.pts, t.nrm, t.nodes, t.pts16, (int)t.n, t.L, t.obb}; }

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
cudaError_t estimate_normals(const TargetDev *t, int k, const double viewpoint[3], float *out_dev, cudaStream_t s,
                             int *overflow_out);
cudaError_t build_fp16_storage(TargetDev *t, cudaStream_t s);
// Source points in Morton order (and, when n_dev is given, their normals in the
// same order into nrm_out; a normal that is neither zero nor unit length within
// 1e-3 counts as bad input).
cudaError_t prepare_source(const float *p_dev, int64_t m, cudaStream_t s, float4 *src_out,
                           float lo[3], float hi[3], int *bad_input, const float *n_dev = nullptr,
                           float4 *nrm_out = nullptr);
cudaError_t launch_closest(const TargetDev *t, const float *p_dev, int64_t m, const double T[12],
                           int64_t *idx, double *d2, cudaStream_t s);
// One device step: the closest-point search kernel (query tiles, or one query
// per warp for search == FRICP_SEARCH_QUERY), then the accumulate/solve
// kernel. When `mid` is given it is recorded between the two.
cudaError_t launch_step(const StepArgs &a, int variant, int prec, int ntiles, cudaStream_t s,
                        cudaEvent_t mid = nullptr, int search = FRICP_SEARCH_QUERY);
cudaError_t launch_setup_eval_xi(PairState *st, const double *T_normalized12, cudaStream_t s);
// Median of n non-negative doubles (the mean of the two middle order
// statistics, exact) by a grid-wide 8-bit radix select; `scratch` holds
// kMedianScratchBytes of device memory, the result lands in *out_dev.
constexpr int kMedianScratchBytes = 4096;
cudaError_t launch_median(const double *v, int n, void *scratch, double *out_dev, cudaStream_t s);
// After a first pass run with init_median_ext: nu_max from the median at
// *median_dev and the first nu stage (start_after_init).
cudaError_t launch_after_init(PairState *st, const double *median_dev, cudaStream_t s);

}  // namespace fricp
