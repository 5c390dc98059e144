// Device state machine of Algorithm 1 (Welsch point-to-point ICP, and with
// psi -> squared distance, unit weights and one stage, the accelerated
// point-to-point "Fast ICP") and Algorithm 2 (Welsch point-to-plane ICP).
//
// Every fused step kernel evaluates one transform (closest points, residuals,
// weights, energy and the reduced sums of the alignment problem); its last
// block then calls solver_step() on one thread, which consumes those sums,
// takes every decision the algorithm makes between two correspondence passes
// (energy safeguard, alignment / Gauss-Newton solve, convergence test,
// Anderson step, line search, nu stage change) and writes the transform the
// next pass must evaluate. The iteration counter k of the paper only appears
// through k - k_start, kept as n_body + 1.
#pragma once

#include "fricp_internal.cuh"
#include "linalg.cuh"

namespace fricp {

FRICP_HD inline void copy_n(double *dst, const double *src, int n) {
    for (int i = 0; i < n; ++i) dst[i] = src[i];
}

// Next pass evaluates the normalised transform T (R row-major, t): the pass
// works in caller units, x = R p + t_o with t_o = t / s + c - R c.
FRICP_HD inline void request_eval_T(PairState *st, const double T[12], int counts) {
    for (int i = 0; i < 9; ++i) st->Re[i] = T[i];
    for (int r = 0; r < 3; ++r) {
        const double Rc = T[3 * r] * st->c[0] + T[3 * r + 1] * st->c[1] + T[3 * r + 2] * st->c[2];
        st->te[r] = T[9 + r] / st->s + st->c[r] - Rc;
    }
    st->eval_counts = counts;
}

FRICP_HD inline void request_eval_xi(PairState *st, const double xi[6], int counts) {
    double T[12];
    se3_exp(xi, T);
    copy_n(st->xeval, xi, 6);
    request_eval_T(st, T, counts);
}

__device__ inline void push_trace(PairState *st, double *trace, double E) {
    if (trace != nullptr && st->trace_len < st->trace_cap) trace[st->trace_len] = E;
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
__device__ inline void anderson_step(PairState *st, int mk, double wrot, double x_out[6]) {
    const int nw = st->hlen - 1;
    copy_n(x_out, st->Gh[nw], 6);
    if (mk <= 0) return;
    double D[6][kMaxM], f[6], theta[kMaxM];
    for (int i = 0; i < 6; ++i) {
        const double wi = (i < 3) ? wrot : 1.0;
        f[i] = wi * st->Fh[nw][i];
        for (int j = 1; j <= mk; ++j) D[i][j - 1] = wi * (st->Fh[nw - j + 1][i] - st->Fh[nw - j][i]);
    }
    if (!anderson_lstsq(D, f, mk, theta)) return;
    for (int j = 1; j <= mk; ++j)
        for (int i = 0; i < 6; ++i) x_out[i] -= theta[j - 1] * (st->Gh[nw - j + 1][i] - st->Gh[nw - j][i]);
}

// ---------------------------------------------------------------------------
// Algorithm 1
// ---------------------------------------------------------------------------

// Alignment step (Eq. 4 / Eq. 12) from the reduced sums, in normalised units.
// Sums are over p~ = p - c and q~ = q - c (caller units): S[0] = sum w,
// S[1..3] = sum w p~, S[4..6] = sum w q~, S[7..15] = sum w p~ q~^T, S[16] = E.
__device__ inline bool align_from_sums(const PairState *st, const double *S, double T[12]) {
    const double W = S[0];
    if (!(W > 0.0) || !isfinite(W)) return false;
    double pb[3], qb[3], H[9];
    for (int a = 0; a < 3; ++a) {
        pb[a] = S[1 + a] / W;
        qb[a] = S[4 + a] / W;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) H[3 * a + b] = S[7 + 3 * a + b] - W * pb[a] * qb[b];
    if (!procrustes_rotation(H, T)) return false;
    for (int r = 0; r < 3; ++r) {
        const double Rp = T[3 * r] * pb[0] + T[3 * r + 1] * pb[1] + T[3 * r + 2] * pb[2];
        T[9 + r] = st->s * (qb[r] - Rp);
    }
    return true;
}

__device__ inline void p2p_stage_end(PairState *st, int stage_pass_counts) {
    if (st->nu == st->nu_min) {
        finish(st, FRICP_OK);
        return;
    }
    st->nu = fmax(0.5 * st->nu, st->nu_min);
    request_eval_T(st, st->Tk, stage_pass_counts);
    st->phase = PH_STAGE_START;
}

__device__ inline void p2p_continue(PairState *st, double E, const double *S, double *trace) {
    st->E_prev = E;
    push_trace(st, trace, E);
    double Tn[12];
    if (!align_from_sums(st, S, Tn)) {
        finish(st, FRICP_EDEGENERATE);
        return;
    }
    copy_n(st->Tp, Tn, 12);
    double fro = 0.0;
    for (int i = 0; i < 12; ++i) fro += (st->Tk[i] - st->Tp[i]) * (st->Tk[i] - st->Tp[i]);
    if (fro < st->eps * st->eps) {
        p2p_stage_end(st, 0);
        return;
    }
    double g[6], f[6];
    se3_log(st->Tp, g);
    copy_n(st->logTp, g, 6);
    for (int i = 0; i < 6; ++i) f[i] = g[i] - st->logTk[i];   // log T^(k) is cached with T^(k)
    hist_push(st, g, f);
    const int mk = min(st->n_body + 1, st->m);
    double x[6];
    anderson_step(st, mk, 1.4142135623730951, x);
    se3_exp(x, st->Tk);
    copy_n(st->logTk, x, 6);   // log(exp(x)) = x for rotation angles below pi
    st->n_body++;
    request_eval_T(st, st->Tk, 1);
    st->phase = (st->n_body + 1 <= st->max_iters) ? PH_ITER : PH_CAPCHECK;
}

__device__ inline void p2p_step(PairState *st, const double *S, double *trace) {
    const double E = S[kSumsP2P - 1];
    switch (st->phase) {
    case PH_STAGE_START: {
        double Tn[12];
        if (!align_from_sums(st, S, Tn)) {
            finish(st, FRICP_EDEGENERATE);
            return;
        }
        copy_n(st->Tprev, st->Tk, 12);
        copy_n(st->Tp, Tn, 12);
        copy_n(st->Tk, Tn, 12);
        double g[6], f[6];
        se3_log(Tn, g);
        for (int i = 0; i < 6; ++i) f[i] = g[i] - st->logTk[i];   // log T^(k-1), cached
        copy_n(st->logTp, g, 6);
        copy_n(st->logTk, g, 6);
        st->hlen = 0;
        hist_push(st, g, f);
        st->E_prev = INFINITY;
        st->n_body = 0;
        st->stages++;
        request_eval_T(st, st->Tk, 1);
        st->phase = (1 <= st->max_iters) ? PH_ITER : PH_CAPCHECK;
        break;
    }
    case PH_ITER:
        st->iterations++;
        if (E >= st->E_prev) {   // safeguard: revert to the un-accelerated T'
            st->reverts++;
            copy_n(st->Tk, st->Tp, 12);
            copy_n(st->logTk, st->logTp, 6);
            request_eval_T(st, st->Tk, 1);
            st->phase = PH_ITER_REVERTED;
            return;
        }
        if (st->n_body > 0) st->aa_accepted++;
        p2p_continue(st, E, S, trace);
        break;
    case PH_ITER_REVERTED:
        p2p_continue(st, E, S, trace);
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
        p2p_stage_end(st, rev);
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
// row by row), SzB = S[21..26].
__device__ inline bool gn_delta(const double xi[6], const double *S, double d[6]) {
    double K[36], Z[36];
    p2pl_chain(xi, K);
    int t = 0;
    for (int r = 0; r < 6; ++r)
        for (int c = r; c < 6; ++c) {
            Z[6 * r + c] = S[t];
            Z[6 * c + r] = S[t];
            ++t;
        }
    double KZ[36], A[36], g[6];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k) acc += K[6 * r + k] * Z[6 * k + c];
            KZ[6 * r + c] = acc;
        }
    for (int r = 0; r < 6; ++r) {
        for (int c = 0; c < 6; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k) acc += KZ[6 * r + k] * K[6 * c + k];
            A[6 * r + c] = acc;
        }
        double acc = 0.0;
        for (int k = 0; k < 6; ++k) acc += K[6 * r + k] * S[21 + k];
        g[r] = -acc;
    }
    return chol6_solve(A, g, d);
}

__device__ inline void p2pl_stage_end(PairState *st) {
    if (st->nu == st->nu_min) {
        finish(st, FRICP_OK);
        return;
    }
    st->nu = fmax(0.5 * st->nu, st->nu_min);
    st->cap = min(st->cap + 1, st->cap_max);
    request_eval_xi(st, st->xk, 0);
    st->phase = PH_STAGE_START;
}

__device__ inline void p2pl_continue(PairState *st, double E, const double *S, double *trace) {
    st->E_prev = E;
    push_trace(st, trace, E);
    double d[6];
    if (!gn_delta(st->xk, S, d)) {
        finish(st, FRICP_EDEGENERATE);
        return;
    }
    double xs[6], f[6], nrm = 0.0;
    for (int i = 0; i < 6; ++i) {
        xs[i] = st->xk[i] + d[i];
        f[i] = xs[i] - st->xk[i];
        nrm += f[i] * f[i];
    }
    if (sqrt(nrm) < st->eps) {
        p2pl_stage_end(st);
        return;
    }
    hist_push(st, xs, f);
    const int mk = min(st->n_body + 1, st->m);
    double x[6];
    anderson_step(st, mk, 1.0, x);   // Reading: no exp, xi is already the parameter
    copy_n(st->xprev, st->xk, 6);
    copy_n(st->xstar, xs, 6);
    copy_n(st->xk, x, 6);
    st->n_body++;
    request_eval_xi(st, st->xk, 1);
    st->phase = (st->n_body + 1 <= st->cap) ? PH_ITER : PH_CAPCHECK;
}

__device__ inline void ls_trial(PairState *st) {
    double x[6];
    for (int i = 0; i < 6; ++i) x[i] = st->xprev[i] + st->tau * (st->xstar[i] - st->xprev[i]);
    request_eval_xi(st, x, 1);
    st->phase = PH_LS;
}

__device__ inline void ls_finish(PairState *st, double *trace) {
    copy_n(st->xk, st->xbest, 6);
    if (st->capexit)
        p2pl_stage_end(st);
    else
        p2pl_continue(st, st->E_best, st->sys_best, trace);
}

// Alg. 2 line search along xi*^(k) - xi^(k-1), keeping the lowest energy seen.
// Reading: tau halves and l grows after every trial; l_max = max_ls.
__device__ inline void ls_begin(PairState *st, double E, const double *S, int capexit, double *trace) {
    st->E_best = E;
    copy_n(st->xbest, st->xk, 6);
    copy_n(st->sys_best, S, kSumsP2PL);
    st->tau = 1.0;
    st->ls_l = 1;
    st->capexit = capexit;
    if (st->max_ls < 1) {
        ls_finish(st, trace);
        return;
    }
    ls_trial(st);
}

__device__ inline void p2pl_step(PairState *st, const double *S, double *trace) {
    const double E = S[kSumsP2PL - 1];
    switch (st->phase) {
    case PH_STAGE_START: {
        double d[6];
        if (!gn_delta(st->xk, S, d)) {
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
        request_eval_xi(st, st->xk, 1);
        st->phase = (1 <= st->cap) ? PH_ITER : PH_CAPCHECK;
        break;
    }
    case PH_ITER:
        st->iterations++;
        if (E >= st->E_prev) {
            st->reverts++;
            ls_begin(st, E, S, 0, trace);
            return;
        }
        if (st->n_body > 0) st->aa_accepted++;
        p2pl_continue(st, E, S, trace);
        break;
    case PH_CAPCHECK:
        if (E >= st->E_prev) {
            st->reverts++;
            ls_begin(st, E, S, 1, trace);
            return;
        }
        p2pl_stage_end(st);
        break;
    case PH_LS:
        st->ls_trials++;
        if (E < st->E_best) {
            st->E_best = E;
            copy_n(st->xbest, st->xeval, 6);
            copy_n(st->sys_best, S, kSumsP2PL);
        }
        if (E < st->E_prev || st->ls_l >= st->max_ls) {
            ls_finish(st, trace);
        } else {
            st->tau *= 0.5;
            st->ls_l++;
            ls_trial(st);
        }
        break;
    default:
        finish(st, FRICP_EINVAL);
    }
}

// Set the nu range after the initial pass (Sec. 4.3 / Sec. 5): nu_max = 3 x
// median residual at T0 unless given; nu_min was fixed by the host (given, or
// from the target's six-neighbour statistic) and clamped; a nu_max below
// nu_min collapses to a single stage at nu_min.
static __device__ __noinline__ void start_after_init(PairState *st, double median) {
    if (!st->nu_max_given) st->nu_max = 3.0 * median;
    st->nu_max = fmax(st->nu_max, st->nu_min);
    st->nu = st->nu_max;
    st->cap = st->cap_first;
    st->phase = PH_STAGE_START;
    st->eval_counts = 0;   // the stage-start pass re-uses the correspondences at T0
}

static __device__ __noinline__ void solver_step(PairState *st, const double *S, double *trace) {
    st->device_steps++;
    if (st->eval_counts) st->corr_passes++;
    if (st->phase == PH_EVAL) {
        st->eval_out[0] = S[fricp::variant_p2pl(st->variant) ? kSumsP2PL - 1 : kSumsP2P - 1];
        int ok;
        if (fricp::variant_p2pl(st->variant)) {
            double d[6];
            ok = gn_delta(st->xeval, S, d);
            for (int i = 0; i < 6; ++i) st->eval_out[1 + i] = st->xeval[i] + d[i];
        } else {
            double T[12];
            ok = align_from_sums(st, S, T);
            for (int i = 0; i < 12; ++i) st->eval_out[1 + i] = T[i];
        }
        const int K = fricp::variant_p2pl(st->variant) ? kSumsP2PL : kSumsP2P;
        for (int k = 0; k < K; ++k) st->eval_out[16 + k] = S[k];
        st->status = ok ? FRICP_OK : FRICP_EDEGENERATE;
        st->phase = PH_DONE;
        st->done = 1;
        return;
    }
    if (fricp::variant_p2pl(st->variant))
        p2pl_step(st, S, trace);
    else
        p2p_step(st, S, trace);
}

}  // namespace fricp
