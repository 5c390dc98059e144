// C ABI of libfricp (declared in include/fricp.h): argument checking, device
// buffers, the host loop that replays fused steps until the device-side state
// machine reports done, and the conversion of the result to caller units.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "fricp_internal.cuh"
#include "linalg.cuh"
#include "solver.cuh"

using fricp::PairState;
using fricp::TargetDev;

struct fricp_target {
    TargetDev d;
};

namespace fricp {
Counters &counters() {
    thread_local Counters c{0, 0, 0};
    return c;
}
}  // namespace fricp

namespace {

using fricp::counters;

thread_local std::string g_err;

fricp_status fail(fricp_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

fricp_status cuda_fail(cudaError_t e, const char *where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return FRICP_ECUDA;
}

// One non-blocking stream per host thread: graphs can be captured on it, and it
// is ordered after / before the caller's stream with events.
cudaStream_t work_stream() {
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

int *pinned_flag() {
    thread_local int *p = nullptr;
    if (p == nullptr) cudaMallocHost(&p, 64);
    return p;
}

bool host_finite(const float *x, int64_t n3) {
    for (int64_t i = 0; i < n3; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

fricp_status check_params(const fricp_params *p) {
    if (p->variant < FRICP_P2P_AA || p->variant > FRICP_P2PL_WELSCH_AA) return fail(FRICP_EINVAL, "unknown variant");
    if (p->anderson_m < 0 || p->anderson_m > fricp::kMaxM) return fail(FRICP_EINVAL, "anderson_m must be in 0..5");
    if (p->max_iters < 1 || p->p2pl_iters_first < 1 || p->p2pl_iters_cap < p->p2pl_iters_first)
        return fail(FRICP_EINVAL, "iteration caps must be >= 1 and cap >= first");
    if (p->max_line_search < 0) return fail(FRICP_EINVAL, "max_line_search must be >= 0");
    if (!(p->eps > 0.0)) return fail(FRICP_EINVAL, "eps must be > 0");
    if (!(p->nu_min_floor > 0.0)) return fail(FRICP_EINVAL, "nu_min_floor must be > 0");
    if (p->steps_per_sync < 1 || p->steps_per_sync > 4096) return fail(FRICP_EINVAL, "steps_per_sync in 1..4096");
    if (p->max_steps < 1) return fail(FRICP_EINVAL, "max_steps must be >= 1");
    if (!(p->timeout_s > 0.0)) return fail(FRICP_EINVAL, "timeout_s must be > 0");
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

fricp_status stage_input(const float *x, int64_t n, int on_device, cudaStream_t s, DevInput *out, const char *what) {
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

fricp_status wait_event(cudaEvent_t ev, std::chrono::steady_clock::time_point deadline) {
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
void normalisation(const TargetDev &t, const float plo[3], const float phi[3], double *s, double c[3]) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double lo = std::fmin((double)plo[a], (double)t.lo[a]);
        const double hi = std::fmax((double)phi[a], (double)t.hi[a]);
        d2 += (hi - lo) * (hi - lo);
        c[a] = t.centroid[a];
    }
    *s = d2 > 0.0 ? 1.0 / std::sqrt(d2) : 1.0;
}

void to_normalised(const double *T0, double s, const double c[3], double Tn[12]) {
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

void to_caller(const double Tn[12], double s, const double c[3], double R[9], double t[3]) {
    for (int i = 0; i < 9; ++i) R[i] = Tn[i];
    for (int r = 0; r < 3; ++r) {
        const double Rc = Tn[3 * r] * c[0] + Tn[3 * r + 1] * c[1] + Tn[3 * r + 2] * c[2];
        t[r] = Tn[9 + r] / s + c[r] - Rc;
    }
}

struct Graph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t g = nullptr;
    ~Graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
    }
};

// Run fused steps until the state machine is done. Returns the status and the
// summed device time of the step launches when timing is requested.
fricp_status run_steps(const fricp::StepArgs &a, int variant, int ntiles, const fricp_params &prm, cudaStream_t s,
                       PairState *st_dev, bool *leak, double *pass_ms) {
    using clock = std::chrono::steady_clock;
    const auto deadline = clock::now() + std::chrono::duration_cast<clock::duration>(
                                             std::chrono::duration<double>(prm.timeout_s));
    int *done_h = pinned_flag();
    cudaEvent_t poll;
    cudaEventCreateWithFlags(&poll, cudaEventDisableTiming);
    const int chunk = prm.steps_per_sync;
    Graph graph;
    const bool timing = prm.time_passes != 0;
    const bool use_graph = prm.use_graph && !timing;
    std::vector<cudaEvent_t> tev;
    if (timing) {
        tev.resize(2 * chunk);
        for (auto &e : tev) cudaEventCreate(&e);
    }
    fricp_status rs = FRICP_OK;
    cudaError_t e = cudaSuccess;
    if (use_graph) {
        const int64_t before = counters().launches;   // capture records launches, it does not run them
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < chunk; ++k) fricp::launch_step(a, variant, ntiles, s);
            e = cudaStreamEndCapture(s, &graph.g);
        }
        counters().launches = before;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&graph.exec, graph.g, 0);
        if (e != cudaSuccess) rs = cuda_fail(e, "capturing the step graph");
    }
    int64_t steps = 0;
    *pass_ms = 0.0;
    while (rs == FRICP_OK) {
        if (use_graph) {
            e = cudaGraphLaunch(graph.exec, s);
            counters().launches += chunk;
        } else {
            for (int k = 0; k < chunk && e == cudaSuccess; ++k) {
                if (timing) cudaEventRecord(tev[2 * k], s);
                e = fricp::launch_step(a, variant, ntiles, s);
                if (timing) cudaEventRecord(tev[2 * k + 1], s);
            }
        }
        if (e != cudaSuccess) {
            rs = cuda_fail(e, "launching step");
            break;
        }
        steps += chunk;
        e = cudaMemcpyAsync(done_h, &st_dev->done, sizeof(int), cudaMemcpyDeviceToHost, s);
        counters().d2h += sizeof(int);
        if (e == cudaSuccess) e = cudaEventRecord(poll, s);
        if (e != cudaSuccess) {
            rs = cuda_fail(e, "polling");
            break;
        }
        rs = wait_event(poll, deadline);
        if (rs != FRICP_OK) {
            *leak = true;   // steps may still be queued: keep their buffers alive
            break;
        }
        if (timing) {
            for (int k = 0; k < chunk; ++k) {
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, tev[2 * k], tev[2 * k + 1]);
                *pass_ms += ms;
            }
        }
        if (*done_h) break;
        if (steps >= prm.max_steps) {
            rs = fail(FRICP_ETIMEOUT, "step budget exhausted before convergence");
            break;
        }
    }
    for (auto &ev : tev) cudaEventDestroy(ev);
    cudaEventDestroy(poll);
    return rs;
}

PairState initial_state(const fricp_params &prm, int64_t m, int ntiles, double s, const double c[3],
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
    h.nu_max = prm.nu_max > 0.0 ? prm.nu_max : 0.0;
    h.nu_min = nu_min;
    h.E_prev = INFINITY;
    h.cap = prm.p2pl_iters_first;
    return h;
}

}  // namespace

namespace fricp {
const TargetDev *target_dev(const fricp_target *t) { return t ? &t->d : nullptr; }
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace fricp

extern "C" {

int32_t fricp_version(void) { return (1 << 16) | 0; }

void fricp_counters(int64_t *kernel_launches, int64_t *h2d_bytes, int64_t *d2h_bytes, int32_t reset) {
    fricp::Counters &c = counters();
    if (kernel_launches) *kernel_launches = c.launches;
    if (h2d_bytes) *h2d_bytes = c.h2d;
    if (d2h_bytes) *d2h_bytes = c.d2h;
    if (reset) c = fricp::Counters{0, 0, 0};
}

const char *fricp_last_error(void) { return g_err.c_str(); }

fricp_status fricp_params_default(int32_t variant, fricp_params *out) {
    if (out == nullptr) return fail(FRICP_EINVAL, "out is NULL");
    if (variant < FRICP_P2P_AA || variant > FRICP_P2PL_WELSCH_AA) return fail(FRICP_EINVAL, "unknown variant");
    std::memset(out, 0, sizeof(*out));
    out->variant = variant;
    out->anderson_m = 5;
    out->max_iters = 1000;
    out->p2pl_iters_first = 6;
    out->p2pl_iters_cap = 10;
    out->max_line_search = 10;
    out->eps = 1e-5;
    out->nu_max = 0.0;
    out->nu_min = 0.0;
    out->nu_min_floor = 1e-6;
    out->steps_per_sync = 16;
    out->use_graph = 1;
    out->time_passes = 0;
    out->max_steps = 100000;
    out->timeout_s = 600.0;
    return FRICP_OK;
}

fricp_status fricp_target_create(const float *q_xyz, const float *q_normals, int64_t n, int32_t on_device,
                                 void *stream, fricp_target **out) {
    if (out == nullptr || q_xyz == nullptr) return fail(FRICP_EINVAL, "NULL argument");
    *out = nullptr;
    if (n < 1 || n > (int64_t)1 << 30) return fail(FRICP_EINVAL, "n must be in 1..2^30");
    Ordered ord(stream);
    DevInput q, nq;
    fricp_status st = stage_input(q_xyz, n, on_device, ord.work, &q, "q_xyz");
    if (st != FRICP_OK) return st;
    if (q_normals) {
        st = stage_input(q_normals, n, on_device, ord.work, &nq, "q_normals");
        if (st != FRICP_OK) return st;
    }
    fricp_target *t = new (std::nothrow) fricp_target;
    if (!t) return fail(FRICP_ENOMEM, "host allocation");
    std::memset(&t->d, 0, sizeof(t->d));
    int bad = 0;
    cudaError_t e = fricp::build_target(q.ptr, q_normals ? nq.ptr : nullptr, n, ord.work, &t->d, &bad);
    if (e != cudaSuccess || bad) {
        if (t->d.pts) cudaFree(t->d.pts);
        if (t->d.nrm) cudaFree(t->d.nrm);
        if (t->d.nodes) cudaFree(t->d.nodes);
        delete t;
        if (bad) return fail(FRICP_EINVAL, "target has NaN/Inf coordinates or non-unit normals");
        return e == cudaErrorMemoryAllocation ? fail(FRICP_ENOMEM, "device allocation for the target index")
                                              : cuda_fail(e, "building the target index");
    }
    *out = t;
    return FRICP_OK;
}

fricp_status fricp_target_destroy(fricp_target *t) {
    if (t == nullptr) return FRICP_OK;
    cudaDeviceSynchronize();
    if (t->d.pts) cudaFree(t->d.pts);
    if (t->d.nrm) cudaFree(t->d.nrm);
    if (t->d.nodes) cudaFree(t->d.nodes);
    delete t;
    return FRICP_OK;
}

int64_t fricp_target_size(const fricp_target *t) { return t ? t->d.n : 0; }
int32_t fricp_target_has_normals(const fricp_target *t) { return t ? t->d.has_normals : 0; }

fricp_status fricp_target_nu_min(const fricp_target *t, int32_t variant, double scale, void *stream,
                                 double *nu_min_out) {
    if (!t || !nu_min_out) return fail(FRICP_EINVAL, "NULL argument");
    if (variant == FRICP_P2PL_WELSCH_AA && !t->d.has_normals)
        return fail(FRICP_EUNSUPPORTED, "point-to-plane needs target normals");
    Ordered ord(stream);
    cudaError_t e = fricp::target_nu_stats(const_cast<TargetDev *>(&t->d), ord.work);
    if (e != cudaSuccess) return cuda_fail(e, "nu_min statistics");
    *nu_min_out = variant == FRICP_P2PL_WELSCH_AA ? scale * t->d.H_Q / 6.0 : scale * t->d.E_Q / (3.0 * std::sqrt(3.0));
    return FRICP_OK;
}

fricp_status fricp_closest_points(const fricp_target *t, const float *p_xyz, int64_t m, const double *T,
                                  int64_t *idx_out, double *d2_out, void *stream) {
    if (!t || !p_xyz || !idx_out || !d2_out) return fail(FRICP_EINVAL, "NULL argument");
    if (m < 0 || m > (int64_t)1 << 30) return fail(FRICP_EINVAL, "m out of range");
    if (m == 0) return FRICP_OK;
    double T12[12] = {1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0};
    if (T)
        for (int r = 0; r < 3; ++r) {
            for (int k = 0; k < 3; ++k) T12[3 * r + k] = T[4 * r + k];
            T12[9 + r] = T[4 * r + 3];
        }
    const cudaError_t e = fricp::launch_closest(&t->d, p_xyz, m, T12, idx_out, d2_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "closest points");
    return FRICP_OK;
}

fricp_status fricp_register(const fricp_target *t, const float *p_xyz, int64_t m, int32_t on_device,
                            const double *T0, const fricp_params *params, void *stream, fricp_result *out,
                            double *trace, int32_t trace_capacity) {
    const auto wall0 = std::chrono::steady_clock::now();
    if (!t || !p_xyz || !params || !out) return fail(FRICP_EINVAL, "NULL argument");
    if (m < 1 || m > (int64_t)1 << 30) return fail(FRICP_EINVAL, "m must be in 1..2^30");
    if (trace_capacity < 0 || (trace_capacity > 0 && !trace)) return fail(FRICP_EINVAL, "bad trace buffer");
    fricp_status st = check_params(params);
    if (st != FRICP_OK) return st;
    const fricp_params prm = *params;
    if (prm.variant == FRICP_P2PL_WELSCH_AA && !t->d.has_normals)
        return fail(FRICP_EUNSUPPORTED, "point-to-plane needs target normals");
    if (T0)
        for (int i = 0; i < 16; ++i)
            if (!std::isfinite(T0[i])) return fail(FRICP_EINVAL, "T0 has NaN or Inf");
    std::memset(out, 0, sizeof(*out));
    Ordered ord(stream);
    const cudaStream_t s = ord.work;
    DevInput p;
    st = stage_input(p_xyz, m, on_device, s, &p, "p_xyz");
    if (st != FRICP_OK) return st;

    const int ntiles = (int)((m + fricp::kBlock - 1) / fricp::kBlock);
    const bool robust = prm.variant != FRICP_P2P_AA;
    DevBuf<float4> src;
    DevBuf<PairState> st_dev;
    DevBuf<double> partial, resid, trace_dev;
    DevBuf<int> prev, queue;
    if (src.alloc(m, s) != cudaSuccess || st_dev.alloc(1, s) != cudaSuccess || prev.alloc(m, s) != cudaSuccess ||
        queue.alloc(m, s) != cudaSuccess || partial.alloc((size_t)ntiles * fricp::kMaxSums, s) != cudaSuccess ||
        resid.alloc(robust ? m : 1, s) != cudaSuccess || trace_dev.alloc(trace_capacity, s) != cudaSuccess)
        return fail(FRICP_ENOMEM, "device allocation for the registration");
    float plo[3], phi[3];
    int bad = 0;
    cudaError_t e = fricp::prepare_source(p.ptr, m, s, src.p, plo, phi, &bad);
    if (e != cudaSuccess) return cuda_fail(e, "preparing the source");
    if (bad) return fail(FRICP_EINVAL, "p_xyz has NaN or Inf");

    double scale, c[3];
    normalisation(t->d, plo, phi, &scale, c);
    double nu_min = 1.0;
    if (robust) {
        if (prm.nu_min > 0.0) {
            nu_min = prm.nu_min;
        } else {
            e = fricp::target_nu_stats(const_cast<TargetDev *>(&t->d), s);
            if (e != cudaSuccess) return cuda_fail(e, "nu_min statistics");
            nu_min = prm.variant == FRICP_P2PL_WELSCH_AA ? scale * t->d.H_Q / 6.0
                                                         : scale * t->d.E_Q / (3.0 * std::sqrt(3.0));
        }
        nu_min = std::fmax(nu_min, prm.nu_min_floor);
    }
    PairState h = initial_state(prm, m, ntiles, scale, c, nu_min, trace_capacity);
    double T0n[12];
    to_normalised(T0, scale, c, T0n);
    if (prm.variant == FRICP_P2PL_WELSCH_AA) {
        fricp::se3_log(T0n, h.xk);
        fricp::request_eval_xi(&h, h.xk, 1);
    } else {
        fricp::copy_n(h.Tk, T0n, 12);
        fricp::se3_log(h.Tk, h.logTk);
        fricp::request_eval_T(&h, h.Tk, 1);
    }
    if (robust) {
        h.phase = fricp::PH_INIT;
    } else {
        h.phase = fricp::PH_STAGE_START;
        h.nu = h.nu_max = h.nu_min = 1.0;
    }
    e = cudaMemcpyAsync(st_dev.p, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the solver state");
    counters().h2d += sizeof(h);
    e = cudaMemsetAsync(prev.p, 0xff, sizeof(int) * m, s);   // no correspondence yet
    if (e != cudaSuccess) return cuda_fail(e, "clearing the correspondence buffer");

    fricp::StepArgs a;
    a.st = st_dev.p;
    a.ix = fricp::make_index(t->d);
    a.src = src.p;
    a.prev = prev.p;
    a.queue = queue.p;
    a.partial = partial.p;
    a.resid = resid.p;
    a.trace = trace_capacity > 0 ? trace_dev.p : nullptr;
    bool leak = false;
    double pass_ms = 0.0;
    st = run_steps(a, prm.variant, ntiles, prm, s, st_dev.p, &leak, &pass_ms);
    if (leak) {
        src.leak = st_dev.leak = partial.leak = resid.leak = trace_dev.leak = prev.leak = queue.leak = true;
        p.owned = nullptr;
    }
    if (st != FRICP_OK && st != FRICP_ETIMEOUT) return st;

    PairState r;
    if (!leak) {
        e = cudaMemcpyAsync(&r, st_dev.p, sizeof(r), cudaMemcpyDeviceToHost, s);
        counters().d2h += sizeof(r);
        if (e == cudaSuccess && trace_capacity > 0) {
            e = cudaMemcpyAsync(trace, trace_dev.p, sizeof(double) * trace_capacity, cudaMemcpyDeviceToHost, s);
            counters().d2h += (int64_t)sizeof(double) * trace_capacity;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "reading the result");
    } else {
        return st;
    }
    double Tn[12];
    if (prm.variant == FRICP_P2PL_WELSCH_AA)
        fricp::se3_exp(r.xk, Tn);
    else
        fricp::copy_n(Tn, r.Tk, 12);
    to_caller(Tn, scale, c, out->R, out->t);
    out->status = r.status;
    out->iterations = r.iterations;
    out->corr_passes = r.corr_passes;
    out->aa_accepted = r.aa_accepted;
    out->reverts = r.reverts;
    out->line_search_trials = r.ls_trials;
    out->stages = r.stages;
    out->device_steps = r.device_steps;
    out->trace_len = r.trace_len < trace_capacity ? r.trace_len : trace_capacity;
    out->nu_max = r.nu_max;
    out->nu_min = r.nu_min;
    out->final_energy = r.final_energy;
    out->scale = scale;
    for (int a3 = 0; a3 < 3; ++a3) out->center[a3] = c[a3];
    out->pass_ms = pass_ms;
    out->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    return st;
}

fricp_status fricp_eval_pass(const fricp_target *t, const float *p_xyz, int64_t m, int32_t on_device,
                             int32_t variant, const double *T_normalized, double nu, double scale,
                             const double *center, void *stream, double *out) {
    if (!t || !p_xyz || !T_normalized || !out) return fail(FRICP_EINVAL, "NULL argument");
    if (m < 1 || m > (int64_t)1 << 30) return fail(FRICP_EINVAL, "m must be in 1..2^30");
    if (variant < FRICP_P2P_AA || variant > FRICP_P2PL_WELSCH_AA) return fail(FRICP_EINVAL, "unknown variant");
    if (variant == FRICP_P2PL_WELSCH_AA && !t->d.has_normals)
        return fail(FRICP_EUNSUPPORTED, "point-to-plane needs target normals");
    if (!(scale > 0.0)) return fail(FRICP_EINVAL, "scale must be > 0");
    if (variant != FRICP_P2P_AA && !(nu > 0.0)) return fail(FRICP_EINVAL, "nu must be > 0");
    Ordered ord(stream);
    const cudaStream_t s = ord.work;
    DevInput p;
    fricp_status st = stage_input(p_xyz, m, on_device, s, &p, "p_xyz");
    if (st != FRICP_OK) return st;
    const int ntiles = (int)((m + fricp::kBlock - 1) / fricp::kBlock);
    DevBuf<float4> src;
    DevBuf<PairState> st_dev;
    DevBuf<double> partial, Tdev;
    DevBuf<int> prev, queue;
    if (src.alloc(m, s) != cudaSuccess || st_dev.alloc(1, s) != cudaSuccess || prev.alloc(m, s) != cudaSuccess ||
        queue.alloc(m, s) != cudaSuccess || partial.alloc((size_t)ntiles * fricp::kMaxSums, s) != cudaSuccess ||
        Tdev.alloc(12, s) != cudaSuccess)
        return fail(FRICP_ENOMEM, "device allocation");
    float plo[3], phi[3];
    int bad = 0;
    cudaError_t e = fricp::prepare_source(p.ptr, m, s, src.p, plo, phi, &bad);
    if (e != cudaSuccess) return cuda_fail(e, "preparing the source");
    if (bad) return fail(FRICP_EINVAL, "p_xyz has NaN or Inf");
    fricp_params prm;
    fricp_params_default(variant, &prm);
    const double c[3] = {center ? center[0] : 0.0, center ? center[1] : 0.0, center ? center[2] : 0.0};
    PairState h = initial_state(prm, m, ntiles, scale, c, 1.0, 0);
    h.nu = variant == FRICP_P2P_AA ? 1.0 : nu;
    double T12[12];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) T12[3 * r + k] = T_normalized[4 * r + k];
        T12[9 + r] = T_normalized[4 * r + 3];
    }
    e = cudaMemcpyAsync(st_dev.p, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(prev.p, 0xff, sizeof(int) * m, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Tdev.p, T12, sizeof(T12), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = fricp::launch_setup_eval_xi(st_dev.p, Tdev.p, s);
    fricp::StepArgs a;
    a.st = st_dev.p;
    a.ix = fricp::make_index(t->d);
    a.src = src.p;
    a.prev = prev.p;
    a.queue = queue.p;
    a.partial = partial.p;
    a.resid = nullptr;
    a.trace = nullptr;
    if (e == cudaSuccess) e = fricp::launch_step(a, variant, ntiles, s);
    PairState r;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, st_dev.p, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "evaluation pass");
    for (int i = 0; i < 48; ++i) out[i] = r.eval_out[i];
    if (r.status == FRICP_EDEGENERATE) return fail(FRICP_EDEGENERATE, "degenerate alignment problem");
    return FRICP_OK;
}

}  // extern "C"
