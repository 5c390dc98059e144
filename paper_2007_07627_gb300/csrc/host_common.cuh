// Host-side helpers shared by the C-ABI entry points (api.cu, batch.cu):
// error reporting, the library's work stream, staging of caller arrays,
// stream-ordered device buffers, bounded waits, the normalisation of Sec. 6 and
// the initial solver state of one registration.
#pragma once

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "fricp_internal.cuh"
#include "linalg.cuh"
#include "solver.cuh"

namespace fricp {
namespace host {

inline fricp_status fail(fricp_status s, const std::string &msg) {
    set_last_error(msg.c_str());
    return s;
}

inline fricp_status cuda_fail(cudaError_t e, const char *where) {
    set_last_error((std::string(where) + ": " + cudaGetErrorString(e)).c_str());
    return FRICP_ECUDA;
}

// One non-blocking stream per host thread: graphs can be captured on it, and it
// is ordered after / before the caller's stream with events.
inline cudaStream_t work_stream() {
    thread_local cudaStream_t s = nullptr;
    if (s == nullptr) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    return s;
}

struct Ordered {
    cudaStream_t user, work;
    cudaEvent_t ev = nullptr;
    explicit Ordered(void *stream) : user((cudaStream_t)stream), work(work_stream()) {
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaEventRecord(ev, user);
        cudaStreamWaitEvent(work, ev, 0);
    }
    ~Ordered() {
        cudaEventRecord(ev, work);
        cudaStreamWaitEvent(user, ev, 0);
        cudaEventDestroy(ev);
    }
};

inline int *pinned_flag() {
    thread_local int *p = nullptr;
    if (p == nullptr) cudaMallocHost(&p, 64);
    return p;
}

inline bool host_finite(const float *x, int64_t n3) {
    for (int64_t i = 0; i < n3; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

inline fricp_status check_params(const fricp_params *p) {
    if (p->variant < FRICP_P2P_AA || p->variant > FRICP_SYM_WELSCH_AA) return fail(FRICP_EINVAL, "unknown variant");
    if (p->anderson_m < 0 || p->anderson_m > fricp::kMaxM) return fail(FRICP_EINVAL, "anderson_m must be in 0..5");
    if (p->max_iters < 1 || p->p2pl_iters_first < 1 || p->p2pl_iters_cap < p->p2pl_iters_first)
        return fail(FRICP_EINVAL, "iteration caps must be >= 1 and cap >= first");
    if (p->max_line_search < 0) return fail(FRICP_EINVAL, "max_line_search must be >= 0");
    if (!(p->eps > 0.0)) return fail(FRICP_EINVAL, "eps must be > 0");
    if (!(p->nu_min_floor > 0.0)) return fail(FRICP_EINVAL, "nu_min_floor must be > 0");
    if (p->steps_per_sync < 1 || p->steps_per_sync > 4096) return fail(FRICP_EINVAL, "steps_per_sync in 1..4096");
    if (p->max_steps < 1) return fail(FRICP_EINVAL, "max_steps must be >= 1");
    if (p->precision < FRICP_PREC_FP64 || p->precision > FRICP_PREC_FP16_STORAGE)
        return fail(FRICP_EINVAL, "unknown precision");
    if (!(p->timeout_s > 0.0)) return fail(FRICP_EINVAL, "timeout_s must be > 0");
    if (p->search != FRICP_SEARCH_TILE && p->search != FRICP_SEARCH_QUERY) return fail(FRICP_EINVAL, "unknown search");
    return FRICP_OK;
}

// Device copy of a caller array (host or device). Frees what it allocated.
struct DevInput {
    const float *ptr = nullptr;
    float *owned = nullptr;
    cudaStream_t s = nullptr;
    ~DevInput() {
        if (owned) cudaFreeAsync(owned, s);
    }
};

inline fricp_status stage_input(const float *x, int64_t n, int on_device, cudaStream_t s, DevInput *out, const char *what) {
    out->s = s;
    if (on_device) {
        out->ptr = x;
        return FRICP_OK;
    }
    if (!host_finite(x, 3 * n)) return fail(FRICP_EINVAL, std::string(what) + " has NaN or Inf");
    cudaError_t e = cudaMallocAsync(&out->owned, sizeof(float) * 3 * n, s);
    if (e != cudaSuccess) return fail(FRICP_ENOMEM, std::string("device allocation for ") + what);
    e = cudaMemcpyAsync(out->owned, x, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy input to device");
    counters().h2d += (int64_t)sizeof(float) * 3 * n;
    out->ptr = out->owned;
    return FRICP_OK;
}

template <class T>
struct DevBuf {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    bool leak = false;
    cudaError_t alloc(size_t count, cudaStream_t st) {
        s = st;
        return cudaMallocAsync(&p, sizeof(T) * (count > 0 ? count : 1), st);
    }
    ~DevBuf() {
        if (p && !leak) cudaFreeAsync(p, s);
    }
};

inline fricp_status wait_event(cudaEvent_t ev, std::chrono::steady_clock::time_point deadline) {
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return FRICP_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "waiting for device steps");
        if (std::chrono::steady_clock::now() > deadline) return fail(FRICP_ETIMEOUT, "registration timed out");
        std::this_thread::yield();
    }
}

// Normalisation of both sets by one similarity x -> s (x - c): c = centroid of Q,
// s = 1 / diagonal of the bounding box of P u Q (Sec. 6 set-up).
inline void normalisation(const TargetDev &t, const float plo[3], const float phi[3], double *s, double c[3]) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double lo = std::fmin((double)plo[a], (double)t.lo[a]);
        const double hi = std::fmax((double)phi[a], (double)t.hi[a]);
        d2 += (hi - lo) * (hi - lo);
        c[a] = t.centroid[a];
    }
    *s = d2 > 0.0 ? 1.0 / std::sqrt(d2) : 1.0;
}

inline void to_normalised(const double *T0, double s, const double c[3], double Tn[12]) {
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, t[3] = {0, 0, 0};
    if (T0) {
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) R[3 * r + k] = T0[4 * r + k];
            t[r] = T0[4 * r + 3];
        }
    }
    for (int i = 0; i < 9; ++i) Tn[i] = R[i];
    for (int r = 0; r < 3; ++r) {
        const double Rc = R[3 * r] * c[0] + R[3 * r + 1] * c[1] + R[3 * r + 2] * c[2];
        Tn[9 + r] = s * (Rc + t[r] - c[r]);
    }
}

inline void to_caller(const double Tn[12], double s, const double c[3], double R[9], double t[3]) {
    for (int i = 0; i < 9; ++i) R[i] = Tn[i];
    for (int r = 0; r < 3; ++r) {
        const double Rc = Tn[3 * r] * c[0] + Tn[3 * r + 1] * c[1] + Tn[3 * r + 2] * c[2];
        t[r] = Tn[9 + r] / s + c[r] - Rc;
    }
}

// Kernel nodes of a captured graph (what one replay launches).
inline int64_t graph_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int64_t k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

struct Graph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t g = nullptr;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        exec = nullptr;
        g = nullptr;
    }
    ~Graph() { reset(); }
};

inline PairState initial_state(const fricp_params &prm, int64_t m, int ntiles, double s, const double c[3],
                        double nu_min, int trace_cap) {
    PairState h;
    std::memset(&h, 0, sizeof(h));
    h.variant = prm.variant;
    h.m = prm.anderson_m;
    h.max_iters = prm.max_iters;
    h.cap_first = prm.p2pl_iters_first;
    h.cap_max = prm.p2pl_iters_cap;
    h.max_ls = prm.max_line_search;
    h.M = (int)m;
    h.ntiles = ntiles;
    h.trace_cap = trace_cap;
    h.eps = prm.eps;
    h.s = s;
    for (int a = 0; a < 3; ++a) h.c[a] = c[a];
    h.nu_max_given = prm.nu_max > 0.0;
    h.prec = prm.precision;
    h.nu_max = prm.nu_max > 0.0 ? prm.nu_max : 0.0;
    h.nu_min = nu_min;
    h.E_prev = INFINITY;
    h.cap = prm.p2pl_iters_first;
    if (prm.variant == FRICP_P2PL_AA) {   // one stage: its cap is max_iters (the 6..10 caps belong to nu stages)
        h.cap_first = h.cap_max = h.cap = prm.max_iters;
    }
    return h;
}

// Initial state of one registration whose source was packed by prepare_source
// (bounding box plo/phi): the normalisation, nu_min (the paper's rule from the
// target's statistics unless given, floored), the transform T0 in normalised
// units and the first pass requested (PH_INIT for the robust variants, whose
// first pass also yields nu_max). The target's statistics are computed on
// stream s the first time they are needed.
inline fricp_status setup_pair(const TargetDev &t, const fricp_params &prm, int64_t m, const float plo[3],
                               const float phi[3], const double *T0, int trace_cap, cudaStream_t s, PairState *h,
                               double *scale, double c[3]) {
    normalisation(t, plo, phi, scale, c);
    if (prm.precision == FRICP_PREC_FP16_STORAGE && t.pts16 == nullptr) {
        const cudaError_t e = build_fp16_storage(const_cast<TargetDev *>(&t), s);
        if (e != cudaSuccess) return cuda_fail(e, "FP16 target storage");
    }
    const bool robust = fricp::variant_robust(prm.variant);
    double nu_min = 1.0;
    if (robust) {
        if (prm.nu_min > 0.0) {
            nu_min = prm.nu_min;
        } else {
            const cudaError_t e = target_nu_stats(const_cast<TargetDev *>(&t), s);
            if (e != cudaSuccess) return cuda_fail(e, "nu_min statistics");
            nu_min = fricp::variant_p2pl(prm.variant) ? *scale * t.H_Q / 6.0 : *scale * t.E_Q / (3.0 * std::sqrt(3.0));
        }
        nu_min = std::fmax(nu_min, prm.nu_min_floor);
    }
    const int ntiles = (int)((m + kBlock - 1) / kBlock);
    *h = initial_state(prm, m, ntiles, *scale, c, nu_min, trace_cap);
    double T0n[12];
    to_normalised(T0, *scale, c, T0n);
    std::vector<double> sh(kTeamScratch);
    const Team tm{sh.data()};   // the solver's algebra, as a team of one lane
    if (fricp::variant_p2pl(prm.variant)) {
        log_state_T(tm, T0n, h->xk);
        request_eval_xi(tm, h, h->xk, 1);
    } else {
        copy_n(h->Tk, T0n, 12);
        log_state_T(tm, h->Tk, h->logTk);
        request_eval_state_T(tm, h, h->Tk, 1);
    }
    if (robust) {
        h->phase = PH_INIT;
    } else {
        h->phase = PH_STAGE_START;
        h->nu = h->nu_max = h->nu_min = 1.0;
    }
    set_head_cache_serial(h);
    return FRICP_OK;
}

// Caller-facing result from a registration's final state.
inline void fill_result(const PairState &r, int variant, double scale, const double c[3], int trace_cap,
                        fricp_result *out) {
    double Tn[12];
    if (fricp::variant_p2pl(variant)) {
        std::vector<double> sh(kTeamScratch);
        se3_exp(Team{sh.data()}, r.xk, sh.data(), sh.data() + 12);
        copy_n(Tn, sh.data(), 12);
    } else {
        copy_n(Tn, r.Tk, 12);
    }
    to_caller(Tn, scale, c, out->R, out->t);
    out->status = r.nn_overflow ? FRICP_EOVERFLOW : r.status;
    out->iterations = r.iterations;
    out->corr_passes = r.corr_passes;
    out->aa_accepted = r.aa_accepted;
    out->reverts = r.reverts;
    out->line_search_trials = r.ls_trials;
    out->stages = r.stages;
    out->device_steps = r.device_steps;
    out->trace_len = r.trace_len < trace_cap ? r.trace_len : trace_cap;
    out->nu_max = r.nu_max;
    out->nu_min = r.nu_min;
    out->final_energy = r.final_energy;
    out->scale = scale;
    for (int a = 0; a < 3; ++a) out->center[a] = c[a];
}

}  // namespace host
}  // namespace fricp
