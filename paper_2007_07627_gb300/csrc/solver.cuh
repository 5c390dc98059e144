// Device state machine of Algorithm 1 (Welsch point-to-point ICP, and with
// psi -> squared distance, unit weights and one stage, the accelerated
// point-to-point "Fast ICP") and Algorithm 2 (Welsch point-to-plane ICP).
//
// Every fused step kernel evaluates one transform (closest points, residuals,
// weights, energy and the reduced sums of the alignment problem); one warp of
// its last block then calls solver_step() as a Team (linalg.cuh), which
// consumes those sums, takes every decision the algorithm makes between two
// correspondence passes (energy safeguard, alignment / Gauss-Newton solve,
// convergence test, Anderson step, line search, nu stage change) and writes the
// transform the next pass must evaluate. The iteration counter k of the paper
// only appears through k - k_start, kept as n_body + 1.
//
// Every lane of the team runs the state machine on its own copy of the state
// (so no lane ever reads a value another lane wrote to it); the copies are
// identical, and the lanes write them back word by word. Matrices shared
// between the lanes go through the team scratch.
#pragma once

#include "fricp_internal.cuh"
#include "linalg.cuh"

namespace fricp {

// Team scratch of one solver step (offsets in doubles): the transform of the
// step (12), a second transform (12), the translation of a requested pass (3),
// the Anderson result (6), the Anderson columns and their reciprocals (44) and
// the work area of the alignment / Gauss-Newton solve.
constexpr int kShT = 0, kShT2 = 12, kShTe = 24, kShX = 28, kShD = 40, kShW = 96;
static_assert(kShW + 280 <= kTeamScratch, "team scratch");

FRICP_HD inline void copy_n(double *dst, const double *src, int n) {
    for (int i = 0; i < n; ++i) dst[i] = src[i];
}

// What every block of the next pass derives from Re, te and nu, computed once
// where they change instead of in each block: the float splits hi + lo of Re and
// te (the double-float transform of the search), 1 / (2 nu^2), and the Welsch cap
// radius^2 in caller units, (d_n / s)^2 with d_n^2 / (2 nu^2) = kWelschCut.
FRICP_HD inline void head_scalars(PairState *st) {
    if (st->hnu == st->nu && st->nu > 0.0) return;   // nu changes only at a stage boundary
    st->hnu = st->nu;
    st->hinv2nu2 = st->nu > 0.0 ? 1.0 / (2.0 * st->nu * st->nu) : 0.0;
    const double cut2 = st->nu > 0.0 ? kWelschCut * 2.0 * st->nu * st->nu / (st->s * st->s) : 0.0;
    st->hcut2 = (cut2 > 0.0 && cut2 < 3.0e38) ? (float)(cut2 * (1.0 + 1e-5)) : INFINITY;
}

FRICP_HD inline void set_head_cache_serial(PairState *st) {
    for (int i = 0; i < 9; ++i) split_double(st->Re[i], st->hRh[i], st->hRl[i]);
    for (int r = 0; r < 3; ++r) split_double(st->te[r], st->hth[r], st->htl[r]);
    head_scalars(st);
}

// The same by a team: one split per lane, exchanged through the scratch.
FRICP_HD inline void set_head_cache(const Team &tm, PairState *st) {
    float *f = reinterpret_cast<float *>(tm.sh + kShW);   // 24 floats
    tm.sync();
    for (int e = tm.lane(); e < 12; e += tm.size()) {
        float h, l;
        split_double(e < 9 ? st->Re[e] : st->te[e - 9], h, l);
        f[e] = h;
        f[12 + e] = l;
    }
    tm.sync();
    for (int i = 0; i < 9; ++i) {
        st->hRh[i] = f[i];
        st->hRl[i] = f[12 + i];
    }
    for (int r = 0; r < 3; ++r) {
        st->hth[r] = f[9 + r];
        st->htl[r] = f[21 + r];
    }
    head_scalars(st);
    tm.sync();
}

// Next pass evaluates the normalised transform T (scratch: R row-major, t):
// the pass works in caller units, x = R p + t_o with t_o = t / s + c - R c.
FRICP_HD inline void request_eval_T(const Team &tm, PairState *st, const double *T, int counts) {
    double *te = tm.sh + kShTe;
    tm.sync();
    for (int r = tm.lane(); r < 3; r += tm.size()) {
        const double Rc = fma(T[3 * r + 2], st->c[2], fma(T[3 * r + 1], st->c[1], T[3 * r] * st->c[0]));
        te[r] = T[9 + r] / st->s + st->c[r] - Rc;
    }
    tm.sync();
    for (int i = 0; i < 9; ++i) st->Re[i] = T[i];
    for (int r = 0; r < 3; ++r) st->te[r] = te[r];
    copy_n(st->Teval, T, 12);
    st->eval_counts = counts;
    tm.sync();
}

// The same for a transform held in the state (every lane's copy alike).
FRICP_HD inline void request_eval_state_T(const Team &tm, PairState *st, const double Tst[12], int counts) {
    tm.sync();
    t_store<12>(tm, tm.sh + kShT2, Tst);
    tm.sync();
    request_eval_T(tm, st, tm.sh + kShT2, counts);
}

FRICP_HD inline void request_eval_xi(const Team &tm, PairState *st, const double xi[6], int counts) {
    double x[6];
    copy_n(x, xi, 6);
    se3_exp(tm, x, tm.sh + kShT2, tm.sh + kShW);
    copy_n(st->xeval, x, 6);
    request_eval_T(tm, st, tm.sh + kShT2, counts);
}

// log of a transform held in the state.
FRICP_HD inline void log_state_T(const Team &tm, const double Tst[12], double xi[6]) {
    tm.sync();
    t_store<12>(tm, tm.sh + kShT2, Tst);
    tm.sync();
    se3_log(tm, tm.sh + kShT2, xi, tm.sh + kShW);
}

__device__ inline void push_trace(const Team &tm, PairState *st, double *trace, double E) {
    if (tm.lane() == 0 && trace != nullptr && st->trace_len < st->trace_cap) trace[st->trace_len] = E;
    st->trace_len++;
}

__device__ inline void finish(PairState *st, int status) {
    st->final_energy = st->E_prev;
    st->status = status;
    st->phase = PH_DONE;
    st->done = 1;
}

// Append (G^(k), F^(k)) keeping the newest m + 1 entries.
__device__ inline void hist_push(PairState *st, const double g[6], const double f[6]) {
    const int cap = st->m + 1;
    if (st->hlen == cap) {
        for (int j = 1; j < cap; ++j) {
            copy_n(st->Gh[j - 1], st->Gh[j], 6);
            copy_n(st->Fh[j - 1], st->Fh[j], 6);
        }
        st->hlen--;
    }
    copy_n(st->Gh[st->hlen], g, 6);
    copy_n(st->Fh[st->hlen], f, 6);
    st->hlen++;
}

// Anderson step (Sec. 4.1, Eq. 6) with m_k = min(k - k_start, m) columns.
// wrot weights the three rotational rows of the least squares: sqrt(2) makes
// the Euclidean norm of [w; u] equal the Frobenius norm of the 4x4 se(3) matrix
// that Alg. 1 uses; Alg. 2 uses the plain norm of xi (wrot = 1).
__device__ inline void anderson_step(const Team &tm, const PairState *st, int mk, double wrot, double x_out[6]) {
    const int nw = st->hlen - 1;
    copy_n(x_out, st->Gh[nw], 6);
    if (mk <= 0) return;
    double *Dm = tm.sh + kShD, *xo = tm.sh + kShX;
    tm.sync();
    // column c of D (c < mk): F^(k-c) - F^(k-c-1); column kMaxM: f = F^(k)
    for (int c = tm.lane(); c <= kMaxM; c += tm.size()) {
        if (c == kMaxM) {
#pragma unroll
            for (int i = 0; i < 6; ++i) Dm[6 * c + i] = ((i < 3) ? wrot : 1.0) * st->Fh[nw][i];
        } else if (c < mk) {
#pragma unroll
            for (int i = 0; i < 6; ++i)
                Dm[6 * c + i] = ((i < 3) ? wrot : 1.0) * (st->Fh[nw - c][i] - st->Fh[nw - c - 1][i]);
        }
    }
    tm.sync();
    double theta[kMaxM];
    if (!anderson_lstsq(tm, Dm, mk, theta, Dm + 36)) return;
    for (int i = tm.lane(); i < 6; i += tm.size()) {
        double x = st->Gh[nw][i];
#pragma unroll
        for (int j = 1; j <= kMaxM; ++j)
            if (j <= mk) x = fma(-theta[j - 1], st->Gh[nw - j + 1][i] - st->Gh[nw - j][i], x);
        xo[i] = x;
    }
    tm.sync();
    copy_n(x_out, xo, 6);
    tm.sync();
}

// ---------------------------------------------------------------------------
// Algorithm 1
// ---------------------------------------------------------------------------

// Alignment step (Eq. 4 / Eq. 12) from the reduced sums, in normalised units.
// Sums are over p~ = p - c and q~ = q - c (caller units): S[0] = sum w,
// S[1..3] = sum w p~, S[4..6] = sum w q~, S[7..15] = sum w p~ q~^T, S[16] = E.
// T (12) written to scratch. w: 80 doubles of scratch.
__device__ inline bool align_from_sums(const Team &tm, const PairState *st, const double *S, double *T, double *w) {
    const double W = S[0];
    if (!(W > 0.0) || !isfinite(W)) return false;
    double *pq = w, *H = w + 8, *pw = w + 18;   // pq: pbar (3), qbar (3)
    tm.sync();
    for (int e = tm.lane(); e < 6; e += tm.size()) pq[e] = S[1 + e] / W;
    tm.sync();
    for (int e = tm.lane(); e < 9; e += tm.size()) {
        const int a = e / 3, b = e - 3 * a;
        H[e] = fma(-(W * pq[a]), pq[3 + b], S[7 + e]);
    }
    tm.sync();
    if (!procrustes_rotation(tm, H, T, pw)) return false;
    for (int r = tm.lane(); r < 3; r += tm.size()) {
        const double Rp = fma(T[3 * r + 2], pq[2], fma(T[3 * r + 1], pq[1], T[3 * r] * pq[0]));
        T[9 + r] = st->s * (pq[3 + r] - Rp);
    }
    tm.sync();
    return true;
}

__device__ inline void p2p_stage_end(const Team &tm, PairState *st, int stage_pass_counts) {
    if (st->nu == st->nu_min) {
        finish(st, FRICP_OK);
        return;
    }
    st->nu = fmax(0.5 * st->nu, st->nu_min);
    request_eval_state_T(tm, st, st->Tk, stage_pass_counts);
    st->phase = PH_STAGE_START;
}

__device__ inline void p2p_continue(const Team &tm, PairState *st, double E, const double *S, double *trace) {
    st->E_prev = E;
    push_trace(tm, st, trace, E);
    double *T = tm.sh + kShT;
    if (!align_from_sums(tm, st, S, T, tm.sh + kShW)) {
        finish(st, FRICP_EDEGENERATE);
        return;
    }
    copy_n(st->Tp, T, 12);
    double fro = 0.0;
    for (int i = 0; i < 12; ++i) fro = fma(st->Tk[i] - T[i], st->Tk[i] - T[i], fro);
    if (fro < st->eps * st->eps) {
        p2p_stage_end(tm, st, 0);
        return;
    }
    double g[6], f[6];
    se3_log(tm, T, g, tm.sh + kShW);
    copy_n(st->logTp, g, 6);
    for (int i = 0; i < 6; ++i) f[i] = g[i] - st->logTk[i];   // log T^(k) is cached with T^(k)
    hist_push(st, g, f);
    const int mk = min(st->n_body + 1, st->m);
    double x[6];
    anderson_step(tm, st, mk, 1.4142135623730951, x);
    se3_exp(tm, x, T, tm.sh + kShW);
    copy_n(st->Tk, T, 12);
    copy_n(st->logTk, x, 6);   // log(exp(x)) = x for rotation angles below pi
    st->n_body++;
    request_eval_T(tm, st, T, 1);
    st->phase = (st->n_body + 1 <= st->max_iters) ? PH_ITER : PH_CAPCHECK;
}

__device__ inline void p2p_step(const Team &tm, PairState *st, const double *S, double *trace) {
    const double E = S[kSumsP2P - 1];
    switch (st->phase) {
    case PH_STAGE_START: {
        double *T = tm.sh + kShT;
        if (!align_from_sums(tm, st, S, T, tm.sh + kShW)) {
            finish(st, FRICP_EDEGENERATE);
            return;
        }
        copy_n(st->Tprev, st->Tk, 12);
        copy_n(st->Tp, T, 12);
        copy_n(st->Tk, T, 12);
        double g[6], f[6];
        se3_log(tm, T, g, tm.sh + kShW);
        for (int i = 0; i < 6; ++i) f[i] = g[i] - st->logTk[i];   // log T^(k-1), cached
        copy_n(st->logTp, g, 6);
        copy_n(st->logTk, g, 6);
        st->hlen = 0;
        hist_push(st, g, f);
        st->E_prev = INFINITY;
        st->n_body = 0;
        st->stages++;
        request_eval_T(tm, st, T, 1);
        st->phase = (1 <= st->max_iters) ? PH_ITER : PH_CAPCHECK;
        break;
    }
    case PH_ITER:
        st->iterations++;
        if (E >= st->E_prev) {   // safeguard: revert to the un-accelerated T'
            st->reverts++;
            copy_n(st->Tk, st->Tp, 12);
            copy_n(st->logTk, st->logTp, 6);
            request_eval_state_T(tm, st, st->Tk, 1);
            st->phase = PH_ITER_REVERTED;
            return;
        }
        if (st->n_body > 0) st->aa_accepted++;
        p2p_continue(tm, st, E, S, trace);
        break;
    case PH_ITER_REVERTED:
        p2p_continue(tm, st, E, S, trace);
        break;
    case PH_CAPCHECK: {
        // Reading: the iterate carried out of a stage on the cap is energy-checked too.
        int rev = 0;
        if (E >= st->E_prev) {
            st->reverts++;
            copy_n(st->Tk, st->Tp, 12);
            copy_n(st->logTk, st->logTp, 6);
            rev = 1;
        }
        p2p_stage_end(tm, st, rev);
        break;
    }
    default:
        finish(st, FRICP_EINVAL);
    }
}

// ---------------------------------------------------------------------------
// Algorithm 2
// ---------------------------------------------------------------------------

// Gauss-Newton step of Eq. (18) at xi from the reduced sums: with J_i = K z_i,
// sum g J J^T = K Szz K^T and sum g J B = K SzB, and the reading of Eq. (18)
// sum g J J^T xi* = sum g J (J^T xi - B) gives xi* = xi + d with
// (K Szz K^T) d = -K SzB. Szz is the upper triangle of sum g z z^T (21 values,
// row by row), SzB = S[21..26]. w: 280 doubles of scratch.
__device__ inline bool gn_delta(const Team &tm, const double xi[6], const double *S, double d[6], double *w) {
    double *K = w, *Z = w + 36, *KZ = w + 72, *A = w + 108, *g = w + 144, *cw = w + 152;
    p2pl_chain(tm, xi, K, cw);
    for (int e = tm.lane(); e < 36; e += tm.size()) {
        const int r = e / 6, c = e - 6 * r, lo = r < c ? r : c, hi = r < c ? c : r;
        Z[e] = S[6 * lo - lo * (lo - 1) / 2 + (hi - lo)];
    }
    tm.sync();
    for (int e = tm.lane(); e < 36; e += tm.size()) {
        const int r = e / 6, c = e - 6 * r;
        double acc = K[6 * r] * Z[c];
#pragma unroll
        for (int k = 1; k < 6; ++k) acc = fma(K[6 * r + k], Z[6 * k + c], acc);
        KZ[e] = acc;
    }
    tm.sync();
    // lower triangle of K Szz K^T (21 entries) and the right-hand side -K SzB (6)
    for (int e = tm.lane(); e < 27; e += tm.size()) {
        if (e < 21) {
            int r = 0;
            while ((r + 1) * (r + 2) / 2 <= e) ++r;
            const int c = e - r * (r + 1) / 2;
            double acc = KZ[6 * r] * K[6 * c];
#pragma unroll
            for (int k = 1; k < 6; ++k) acc = fma(KZ[6 * r + k], K[6 * c + k], acc);
            A[6 * r + c] = acc;
        } else {
            const int r = e - 21;
            double acc = K[6 * r] * S[21];
#pragma unroll
            for (int k = 1; k < 6; ++k) acc = fma(K[6 * r + k], S[21 + k], acc);
            g[r] = -acc;
        }
    }
    tm.sync();
    return chol6_solve(tm, A, g, d, cw);
}

__device__ inline void p2pl_stage_end(const Team &tm, PairState *st) {
    if (st->nu == st->nu_min) {
        finish(st, FRICP_OK);
        return;
    }
    st->nu = fmax(0.5 * st->nu, st->nu_min);
    st->cap = min(st->cap + 1, st->cap_max);
    request_eval_xi(tm, st, st->xk, 0);
    st->phase = PH_STAGE_START;
}

__device__ inline void p2pl_continue(const Team &tm, PairState *st, double E, const double *S, double *trace) {
    st->E_prev = E;
    push_trace(tm, st, trace, E);
    double d[6];
    if (!gn_delta(tm, st->xk, S, d, tm.sh + kShW)) {
        finish(st, FRICP_EDEGENERATE);
        return;
    }
    double xs[6], f[6], nrm = 0.0;
    for (int i = 0; i < 6; ++i) {
        xs[i] = st->xk[i] + d[i];
        f[i] = xs[i] - st->xk[i];
        nrm = fma(f[i], f[i], nrm);
    }
    if (sqrt(nrm) < st->eps) {
        p2pl_stage_end(tm, st);
        return;
    }
    hist_push(st, xs, f);
    const int mk = min(st->n_body + 1, st->m);
    double x[6];
    anderson_step(tm, st, mk, 1.0, x);   // Reading: no exp, xi is already the parameter
    copy_n(st->xprev, st->xk, 6);
    copy_n(st->xstar, xs, 6);
    copy_n(st->xk, x, 6);
    st->n_body++;
    request_eval_xi(tm, st, st->xk, 1);
    st->phase = (st->n_body + 1 <= st->cap) ? PH_ITER : PH_CAPCHECK;
}

__device__ inline void ls_trial(const Team &tm, PairState *st) {
    double x[6];
    for (int i = 0; i < 6; ++i) x[i] = fma(st->tau, st->xstar[i] - st->xprev[i], st->xprev[i]);
    request_eval_xi(tm, st, x, 1);
    st->phase = PH_LS;
}

__device__ inline void ls_finish(const Team &tm, PairState *st, double *trace) {
    copy_n(st->xk, st->xbest, 6);
    if (st->capexit)
        p2pl_stage_end(tm, st);
    else
        p2pl_continue(tm, st, st->E_best, st->sys_best, trace);
}

// Alg. 2 line search along xi*^(k) - xi^(k-1), keeping the lowest energy seen.
// Reading: tau halves and l grows after every trial; l_max = max_ls.
__device__ inline void ls_begin(const Team &tm, PairState *st, double E, const double *S, int capexit,
                                double *trace) {
    st->E_best = E;
    copy_n(st->xbest, st->xk, 6);
    copy_n(st->sys_best, S, kSumsP2PL);
    st->tau = 1.0;
    st->ls_l = 1;
    st->capexit = capexit;
    if (st->max_ls < 1) {
        ls_finish(tm, st, trace);
        return;
    }
    ls_trial(tm, st);
}

__device__ inline void p2pl_step(const Team &tm, PairState *st, const double *S, double *trace) {
    const double E = S[kSumsP2PL - 1];
    switch (st->phase) {
    case PH_STAGE_START: {
        double d[6];
        if (!gn_delta(tm, st->xk, S, d, tm.sh + kShW)) {
            finish(st, FRICP_EDEGENERATE);
            return;
        }
        copy_n(st->xprev, st->xk, 6);
        double f[6];
        for (int i = 0; i < 6; ++i) {
            st->xstar[i] = st->xk[i] + d[i];
            f[i] = st->xstar[i] - st->xprev[i];
        }
        copy_n(st->xk, st->xstar, 6);
        st->hlen = 0;
        hist_push(st, st->xstar, f);
        st->E_prev = INFINITY;
        st->n_body = 0;
        st->stages++;
        request_eval_xi(tm, st, st->xk, 1);
        st->phase = (1 <= st->cap) ? PH_ITER : PH_CAPCHECK;
        break;
    }
    case PH_ITER:
        st->iterations++;
        if (E >= st->E_prev) {
            st->reverts++;
            ls_begin(tm, st, E, S, 0, trace);
            return;
        }
        if (st->n_body > 0) st->aa_accepted++;
        p2pl_continue(tm, st, E, S, trace);
        break;
    case PH_CAPCHECK:
        if (E >= st->E_prev) {
            st->reverts++;
            ls_begin(tm, st, E, S, 1, trace);
            return;
        }
        p2pl_stage_end(tm, st);
        break;
    case PH_LS:
        st->ls_trials++;
        if (E < st->E_best) {
            st->E_best = E;
            copy_n(st->xbest, st->xeval, 6);
            copy_n(st->sys_best, S, kSumsP2PL);
        }
        if (E < st->E_prev || st->ls_l >= st->max_ls) {
            ls_finish(tm, st, trace);
        } else {
            st->tau *= 0.5;
            st->ls_l++;
            ls_trial(tm, st);
        }
        break;
    default:
        finish(st, FRICP_EINVAL);
    }
}

// Set the nu range after the initial pass (Sec. 4.3 / Sec. 5): nu_max = 3 x
// median residual at T0 unless given; nu_min was fixed by the host (given, or
// from the target's six-neighbour statistic) and clamped; a nu_max below
// nu_min collapses to a single stage at nu_min. One thread.
static __device__ __noinline__ void start_after_init(PairState *st, double median) {
    if (!st->nu_max_given) st->nu_max = 3.0 * median;
    st->nu_max = fmax(st->nu_max, st->nu_min);
    st->nu = st->nu_max;
    st->cap = st->cap_first;
    st->phase = PH_STAGE_START;
    st->eval_counts = 0;   // the stage-start pass re-uses the correspondences at T0
    head_scalars(st);
}

// Each lane's own copy of the state: coalesced loads by the team into the
// scratch, then every lane copies the scratch. Back: word k by lane k mod size.
constexpr int kStateWords = (int)(sizeof(PairState) / sizeof(double));
static_assert(sizeof(PairState) % sizeof(double) == 0 && kShW + kStateWords <= kTeamScratch, "state copy");

__device__ inline void load_state(const Team &tm, const PairState *g, PairState *own) {
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(g);
    unsigned long long *buf = reinterpret_cast<unsigned long long *>(tm.sh + kShW);
    tm.sync();
    for (int k = tm.lane(); k < kStateWords; k += tm.size()) buf[k] = src[k];
    tm.sync();
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(own);
    for (int k = 0; k < kStateWords; ++k) dst[k] = buf[k];
    tm.sync();
}

__device__ inline void store_state(const Team &tm, const PairState *own, PairState *g) {
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(own);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(g);
    for (int k = tm.lane(); k < kStateWords; k += tm.size()) dst[k] = src[k];
}

// The pass just evaluated, for fricp_register_recorded: the transform, nu, the
// energy, the accepted energy it is compared with, and the alignment (Eq. 4 /
// Eq. 12) or Gauss-Newton (Eq. 19) result the reduced sums give. Every lane
// fills its own copy. Uses the team scratch (before the state machine does).
__device__ inline void record_pass(const Team &tm, const PairState *st, const double *S, bool pl,
                                   fricp_step_record *r) {
    r->step = st->device_steps - 1;
    r->phase = st->phase;
    r->nu = st->nu;
    r->E = S[(pl ? kSumsP2PL : kSumsP2P) - 1];
    r->E_prev = st->E_prev;
    copy_n(r->T, st->Teval, 12);
    for (int i = 0; i < 6; ++i) r->xi[i] = pl ? st->xeval[i] : 0.0;
    for (int i = 0; i < 12; ++i) r->result[i] = 0.0;
    if (pl) {
        double d[6];
        if (gn_delta(tm, st->xeval, S, d, tm.sh + kShW))
            for (int i = 0; i < 6; ++i) r->result[i] = st->xeval[i] + d[i];
    } else {
        double *T = tm.sh + kShT;
        if (align_from_sums(tm, st, S, T, tm.sh + kShW)) copy_n(r->result, T, 12);
        tm.sync();
    }
    r->revert = r->accepted = r->stage = r->done = 0;
}

// One solver step by a team (the first kTeamLanes lanes of a warp; tm.sh:
// kTeamScratch doubles of shared memory). S: the reduced sums of the pass just
// evaluated.
static __device__ __noinline__ void solver_step(Team tm, PairState *gst, const double *S, double *trace) {
    PairState own;
    load_state(tm, gst, &own);
    PairState *st = &own;
    st->device_steps++;
    if (st->eval_counts) st->corr_passes++;
    if (st->phase == PH_EVAL) {
        const bool pl = fricp::variant_p2pl(st->variant);
        st->eval_out[0] = S[pl ? kSumsP2PL - 1 : kSumsP2P - 1];
        int ok;
        if (pl) {
            double d[6];
            ok = gn_delta(tm, st->xeval, S, d, tm.sh + kShW);
            for (int i = 0; i < 6; ++i) st->eval_out[1 + i] = st->xeval[i] + d[i];
        } else {
            double *T = tm.sh + kShT;
            ok = align_from_sums(tm, st, S, T, tm.sh + kShW);
            for (int i = 0; i < 12; ++i) st->eval_out[1 + i] = T[i];
        }
        const int K = pl ? kSumsP2PL : kSumsP2P;
        for (int k = 0; k < K; ++k) st->eval_out[16 + k] = S[k];
        st->status = ok ? FRICP_OK : FRICP_EDEGENERATE;
        st->phase = PH_DONE;
        st->done = 1;
    } else {
        const bool pl = fricp::variant_p2pl(st->variant);
        fricp_step_record r;
        const bool rec = st->rec != nullptr && st->rec_len < st->rec_cap;
        if (rec) record_pass(tm, st, S, pl, &r);
        const int rev0 = st->reverts, acc0 = st->aa_accepted;
        if (pl)
            p2pl_step(tm, st, S, trace);
        else
            p2p_step(tm, st, S, trace);
        if (rec) {
            r.revert = st->reverts - rev0;
            r.accepted = st->aa_accepted - acc0;
            r.stage = st->stages;
            r.done = st->done;
            if (tm.lane() == 0) st->rec[st->rec_len] = r;
            st->rec_len++;
        }
    }
    set_head_cache(tm, st);
    st->counter = 0u;   // the next pass's tile and search tickets start over
    st->nn_next = 0u;
    store_state(tm, st, gst);
}

}  // namespace fricp
