// C ABI of libfricp (declared in include/fricp.h): argument checking, device
// buffers, the host loop that replays fused steps until the device-side state
// machine reports done, and the conversion of the result to caller units.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "host_common.cuh"

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
using namespace fricp::host;

thread_local std::string g_err;

// Run fused steps until the state machine is done. Returns the status and the
// summed device time of the step launches when timing is requested.
// init_m > 0: the state starts at an initial pass flagged init_median_ext; it
// runs first, on its own, and its nu_max median over the init_m residuals is
// selected by the whole GPU (launch_median) before the first stage starts
// (launch_after_init) -- the same median the one-block select in the step would
// find.
fricp_status run_steps(const fricp::StepArgs &a, int variant, int ntiles, const fricp_params &prm, cudaStream_t s,
                       PairState *st_dev, bool *leak, double *pass_ms, double *search_ms, int64_t init_m = 0) {
    using clock = std::chrono::steady_clock;
    const int prec = prm.precision;
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
        tev.resize(3 * chunk);
        for (auto &e : tev) cudaEventCreate(&e);
    }
    fricp_status rs = FRICP_OK;
    cudaError_t e = cudaSuccess;
    if (use_graph) {
        const int64_t before = counters().launches;   // capture records launches, it does not run them
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < chunk; ++k) fricp::launch_step(a, variant, prec, ntiles, s, nullptr, prm.search);
            e = cudaStreamEndCapture(s, &graph.g);
        }
        counters().launches = before;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&graph.exec, graph.g, 0);
        if (e != cudaSuccess) rs = cuda_fail(e, "capturing the step graph");
    }
    const int64_t per_replay = use_graph && graph.g ? graph_kernel_nodes(graph.g) : 0;
    int64_t steps = 0;
    *pass_ms = 0.0;
    *search_ms = 0.0;
    DevBuf<double> mscr;
    if (rs == FRICP_OK && init_m > 0) {
        const size_t words = fricp::kMedianScratchBytes / sizeof(double);
        if (mscr.alloc(words + 1, s) != cudaSuccess) {
            rs = fail(FRICP_ENOMEM, "device allocation for the median select");
        } else {
            double *med = mscr.p + words;
            cudaEvent_t iev[3] = {nullptr, nullptr, nullptr};
            if (timing)
                for (auto &ev : iev) cudaEventCreate(&ev);
            if (timing) cudaEventRecord(iev[0], s);
            e = fricp::launch_step(a, variant, prec, ntiles, s, timing ? iev[1] : nullptr, prm.search);
            if (timing) cudaEventRecord(iev[2], s);
            if (e == cudaSuccess) e = fricp::launch_median(a.resid, (int)init_m, mscr.p, med, s);
            if (e == cudaSuccess) e = fricp::launch_after_init(a.st, med, s);
            if (e != cudaSuccess) rs = cuda_fail(e, "launching the initial pass");
            steps = 1;
            if (timing && rs == FRICP_OK && cudaEventSynchronize(iev[2]) == cudaSuccess) {
                float ms = 0.0f, ms_nn = 0.0f;
                cudaEventElapsedTime(&ms, iev[0], iev[2]);
                cudaEventElapsedTime(&ms_nn, iev[0], iev[1]);
                *pass_ms += ms;
                *search_ms += ms_nn;
            }
            if (timing)
                for (auto &ev : iev) cudaEventDestroy(ev);
        }
    }
    while (rs == FRICP_OK) {
        if (use_graph) {
            e = cudaGraphLaunch(graph.exec, s);
            counters().launches += per_replay;
        } else {
            for (int k = 0; k < chunk && e == cudaSuccess; ++k) {
                if (timing) cudaEventRecord(tev[3 * k], s);
                e = fricp::launch_step(a, variant, prec, ntiles, s, timing ? tev[3 * k + 1] : nullptr, prm.search);
                if (timing) cudaEventRecord(tev[3 * k + 2], s);
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
                float ms = 0.0f, ms_nn = 0.0f;
                cudaEventElapsedTime(&ms, tev[3 * k], tev[3 * k + 2]);
                cudaEventElapsedTime(&ms_nn, tev[3 * k], tev[3 * k + 1]);
                *pass_ms += ms;
                *search_ms += ms_nn;
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
    mscr.leak = *leak;
    return rs;
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
    if (variant < FRICP_P2P_AA || variant > FRICP_SYM_WELSCH_AA) return fail(FRICP_EINVAL, "unknown variant");
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
    out->precision = FRICP_PREC_FP64;
    out->search = FRICP_SEARCH_QUERY;
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

fricp_status fricp_estimate_normals(const float *q_xyz, int64_t n, int32_t k, int32_t on_device,
                                    const double *viewpoint, float *normals_out, void *stream) {
    if (!q_xyz || !normals_out) return fail(FRICP_EINVAL, "NULL argument");
    if (n < 1 || n > (int64_t)1 << 30) return fail(FRICP_EINVAL, "n must be in 1..2^30");
    if (k < 3 || k > 32) return fail(FRICP_EINVAL, "k must be in 3..32");
    double v[3] = {0.0, 0.0, 0.0};
    if (viewpoint)
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(viewpoint[a])) return fail(FRICP_EINVAL, "viewpoint has NaN or Inf");
            v[a] = viewpoint[a];
        }
    Ordered ord(stream);
    const cudaStream_t s = ord.work;
    DevInput q;
    fricp_status st = stage_input(q_xyz, n, on_device, s, &q, "q_xyz");
    if (st != FRICP_OK) return st;
    TargetDev t;
    std::memset(&t, 0, sizeof(t));
    int bad = 0;
    cudaError_t e = fricp::build_target(q.ptr, nullptr, n, s, &t, &bad);
    DevBuf<float> out;
    if (e == cudaSuccess && !bad && !on_device && out.alloc(3 * (size_t)n, s) != cudaSuccess)
        e = cudaErrorMemoryAllocation;
    int overflow = 0;
    if (e == cudaSuccess && !bad)
        e = fricp::estimate_normals(&t, k, v, on_device ? normals_out : out.p, s, &overflow);
    if (e == cudaSuccess && !bad && !on_device) {
        e = cudaMemcpyAsync(normals_out, out.p, sizeof(float) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s);
        counters().d2h += (int64_t)sizeof(float) * 3 * n;
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (t.pts) cudaFree(t.pts);
    if (t.nodes) cudaFree(t.nodes);
    if (bad) return fail(FRICP_EINVAL, "q_xyz has NaN or Inf");
    if (e == cudaErrorMemoryAllocation) return fail(FRICP_ENOMEM, "device allocation for the normal estimate");
    if (e != cudaSuccess) return cuda_fail(e, "normal estimate");
    if (overflow) return fail(FRICP_EOVERFLOW, "neighbour search stack overflow");
    return FRICP_OK;
}

fricp_status fricp_target_destroy(fricp_target *t) {
    if (t == nullptr) return FRICP_OK;
    cudaDeviceSynchronize();
    if (t->d.pts) cudaFree(t->d.pts);
    if (t->d.nrm) cudaFree(t->d.nrm);
    if (t->d.nodes) cudaFree(t->d.nodes);
    if (t->d.pts16) cudaFree(t->d.pts16);
    delete t;
    return FRICP_OK;
}

int64_t fricp_target_size(const fricp_target *t) { return t ? t->d.n : 0; }
int32_t fricp_target_has_normals(const fricp_target *t) { return t ? t->d.has_normals : 0; }

fricp_status fricp_target_nu_min(const fricp_target *t, int32_t variant, double scale, void *stream,
                                 double *nu_min_out) {
    if (!t || !nu_min_out) return fail(FRICP_EINVAL, "NULL argument");
    if (fricp::variant_p2pl(variant) && !t->d.has_normals)
        return fail(FRICP_EUNSUPPORTED, "point-to-plane needs target normals");
    Ordered ord(stream);
    cudaError_t e = fricp::target_nu_stats(const_cast<TargetDev *>(&t->d), ord.work);
    if (e != cudaSuccess) return cuda_fail(e, "nu_min statistics");
    *nu_min_out = fricp::variant_p2pl(variant) ? scale * t->d.H_Q / 6.0 : scale * t->d.E_Q / (3.0 * std::sqrt(3.0));
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

}  // extern "C"

namespace {

// fricp_register, with per-pass records when steps_capacity > 0.
fricp_status register_impl(const fricp_target *t, const float *p_xyz, const float *p_normals, int64_t m,
                           int32_t on_device, const double *T0, const fricp_params *params, void *stream,
                           fricp_result *out, double *trace, int32_t trace_capacity, fricp_step_record *steps,
                           int32_t steps_capacity, int32_t *steps_len) {
    const auto wall0 = std::chrono::steady_clock::now();
    if (!t || !p_xyz || !params || !out) return fail(FRICP_EINVAL, "NULL argument");
    if (steps_capacity < 0 || (steps_capacity > 0 && !steps)) return fail(FRICP_EINVAL, "bad steps buffer");
    if (steps_len) *steps_len = 0;
    if (m < 1 || m > (int64_t)1 << 30) return fail(FRICP_EINVAL, "m must be in 1..2^30");
    if (trace_capacity < 0 || (trace_capacity > 0 && !trace)) return fail(FRICP_EINVAL, "bad trace buffer");
    fricp_status st = check_params(params);
    if (st != FRICP_OK) return st;
    const fricp_params prm = *params;
    if (fricp::variant_p2pl(prm.variant) && !t->d.has_normals)
        return fail(FRICP_EUNSUPPORTED, "point-to-plane needs target normals");
    if (fricp::variant_sym(prm.variant) && !p_normals)
        return fail(FRICP_EUNSUPPORTED, "the symmetric objective needs source normals (fricp_register_symmetric)");
    if (!fricp::variant_sym(prm.variant) && p_normals)
        return fail(FRICP_EINVAL, "source normals are used by FRICP_SYM_WELSCH_AA only");
    if (T0)
        for (int i = 0; i < 16; ++i)
            if (!std::isfinite(T0[i])) return fail(FRICP_EINVAL, "T0 has NaN or Inf");
    std::memset(out, 0, sizeof(*out));
    Ordered ord(stream);
    const cudaStream_t s = ord.work;
    DevInput p, pn;
    st = stage_input(p_xyz, m, on_device, s, &p, "p_xyz");
    if (st != FRICP_OK) return st;
    if (p_normals) {
        st = stage_input(p_normals, m, on_device, s, &pn, "p_normals");
        if (st != FRICP_OK) return st;
    }

    const int ntiles = (int)((m + fricp::kBlock - 1) / fricp::kBlock);
    const bool robust = fricp::variant_robust(prm.variant);
    DevBuf<float4> src;
    DevBuf<PairState> st_dev;
    DevBuf<double> partial, resid, trace_dev;
    DevBuf<int> prev;
    if (src.alloc(m, s) != cudaSuccess || st_dev.alloc(1, s) != cudaSuccess || prev.alloc(m, s) != cudaSuccess ||
        partial.alloc((size_t)ntiles * fricp::kMaxSums, s) != cudaSuccess ||
        resid.alloc(robust ? m : 1, s) != cudaSuccess || trace_dev.alloc(trace_capacity, s) != cudaSuccess)
        return fail(FRICP_ENOMEM, "device allocation for the registration");
    DevBuf<fricp_step_record> rec;
    if (steps_capacity > 0 && rec.alloc(steps_capacity, s) != cudaSuccess)
        return fail(FRICP_ENOMEM, "device allocation for the step records");
    DevBuf<float4> src_nrm;
    if (p_normals && src_nrm.alloc(m, s) != cudaSuccess)
        return fail(FRICP_ENOMEM, "device allocation for the source normals");
    float plo[3], phi[3];
    int bad = 0;
    cudaError_t e = fricp::prepare_source(p.ptr, m, s, src.p, plo, phi, &bad, p_normals ? pn.ptr : nullptr,
                                          p_normals ? src_nrm.p : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "preparing the source");
    if (bad) return fail(FRICP_EINVAL, p_normals ? "p_xyz has NaN or Inf, or p_normals a non-unit normal"
                                                 : "p_xyz has NaN or Inf");

    double scale, c[3];
    PairState h;
    st = setup_pair(t->d, prm, m, plo, phi, T0, trace_capacity, s, &h, &scale, c);
    if (st != FRICP_OK) return st;
    if (steps_capacity > 0) {
        h.rec = rec.p;
        h.rec_cap = steps_capacity;
    }
    h.init_median_ext = h.phase == fricp::PH_INIT ? 1 : 0;
    e = cudaMemcpyAsync(st_dev.p, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the solver state");
    counters().h2d += sizeof(h);
    e = cudaMemsetAsync(prev.p, 0xff, sizeof(int) * m, s);   // no correspondence yet
    if (e != cudaSuccess) return cuda_fail(e, "clearing the correspondence buffer");

    fricp::StepArgs a;
    a.st = st_dev.p;
    a.ix = fricp::make_index(t->d);
    a.src = src.p;
    a.src_nrm = p_normals ? src_nrm.p : nullptr;
    a.prev = prev.p;
    a.partial = partial.p;
    a.resid = resid.p;
    a.trace = trace_capacity > 0 ? trace_dev.p : nullptr;
    bool leak = false;
    double pass_ms = 0.0, search_ms = 0.0;
    st = run_steps(a, prm.variant, ntiles, prm, s, st_dev.p, &leak, &pass_ms, &search_ms, h.init_median_ext ? m : 0);
    if (leak) {
        src.leak = st_dev.leak = partial.leak = resid.leak = trace_dev.leak = prev.leak = rec.leak = src_nrm.leak = true;
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
        if (e == cudaSuccess && steps_capacity > 0) {
            const int n = std::min(r.rec_len, steps_capacity);
            if (n > 0) e = cudaMemcpyAsync(steps, rec.p, sizeof(fricp_step_record) * n, cudaMemcpyDeviceToHost, s);
            counters().d2h += (int64_t)sizeof(fricp_step_record) * n;
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (steps_len) *steps_len = n;
        }
        if (e != cudaSuccess) return cuda_fail(e, "reading the result");
    } else {
        return st;
    }
    fill_result(r, prm.variant, scale, c, trace_capacity, out);
    out->pass_ms = pass_ms;
    out->search_ms = search_ms;
    out->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    return st;
}

}  // namespace

extern "C" {

fricp_status fricp_register(const fricp_target *t, const float *p_xyz, int64_t m, int32_t on_device,
                            const double *T0, const fricp_params *params, void *stream, fricp_result *out,
                            double *trace, int32_t trace_capacity) {
    return register_impl(t, p_xyz, nullptr, m, on_device, T0, params, stream, out, trace, trace_capacity, nullptr,
                         0, nullptr);
}

fricp_status fricp_register_recorded(const fricp_target *t, const float *p_xyz, int64_t m, int32_t on_device,
                                     const double *T0, const fricp_params *params, void *stream,
                                     fricp_result *out, double *trace, int32_t trace_capacity,
                                     fricp_step_record *steps, int32_t steps_capacity, int32_t *steps_len) {
    return register_impl(t, p_xyz, nullptr, m, on_device, T0, params, stream, out, trace, trace_capacity, steps,
                         steps_capacity, steps_len);
}

fricp_status fricp_register_symmetric(const fricp_target *t, const float *p_xyz, const float *p_normals, int64_t m,
                                      int32_t on_device, const double *T0, const fricp_params *params,
                                      void *stream, fricp_result *out, double *trace, int32_t trace_capacity,
                                      fricp_step_record *steps, int32_t steps_capacity, int32_t *steps_len) {
    if (!p_normals) return fail(FRICP_EINVAL, "NULL argument");
    if (params && params->variant != FRICP_SYM_WELSCH_AA)
        return fail(FRICP_EINVAL, "fricp_register_symmetric runs FRICP_SYM_WELSCH_AA");
    return register_impl(t, p_xyz, p_normals, m, on_device, T0, params, stream, out, trace, trace_capacity, steps,
                         steps_capacity, steps_len);
}

fricp_status fricp_eval_pass(const fricp_target *t, const float *p_xyz, int64_t m, int32_t on_device,
                             int32_t variant, const double *T_normalized, double nu, double scale,
                             const double *center, void *stream, double *out) {
    if (!t || !p_xyz || !T_normalized || !out) return fail(FRICP_EINVAL, "NULL argument");
    if (m < 1 || m > (int64_t)1 << 30) return fail(FRICP_EINVAL, "m must be in 1..2^30");
    if (variant == FRICP_SYM_WELSCH_AA)
        return fail(FRICP_EUNSUPPORTED, "the symmetric objective needs source normals (fricp_register_symmetric)");
    if (variant < FRICP_P2P_AA || variant > FRICP_P2PL_AA) return fail(FRICP_EINVAL, "unknown variant");
    if (fricp::variant_p2pl(variant) && !t->d.has_normals)
        return fail(FRICP_EUNSUPPORTED, "point-to-plane needs target normals");
    if (!(scale > 0.0)) return fail(FRICP_EINVAL, "scale must be > 0");
    if (fricp::variant_robust(variant) && !(nu > 0.0)) return fail(FRICP_EINVAL, "nu must be > 0");
    Ordered ord(stream);
    const cudaStream_t s = ord.work;
    DevInput p;
    fricp_status st = stage_input(p_xyz, m, on_device, s, &p, "p_xyz");
    if (st != FRICP_OK) return st;
    const int ntiles = (int)((m + fricp::kBlock - 1) / fricp::kBlock);
    DevBuf<float4> src;
    DevBuf<PairState> st_dev;
    DevBuf<double> partial, Tdev;
    DevBuf<int> prev;
    if (src.alloc(m, s) != cudaSuccess || st_dev.alloc(1, s) != cudaSuccess || prev.alloc(m, s) != cudaSuccess ||
        partial.alloc((size_t)ntiles * fricp::kMaxSums, s) != cudaSuccess ||
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
    h.nu = fricp::variant_robust(variant) ? nu : 1.0;
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
    a.partial = partial.p;
    a.resid = nullptr;
    a.trace = nullptr;
    if (e == cudaSuccess) e = fricp::launch_step(a, variant, fricp::PREC_FP64, ntiles, s, nullptr, FRICP_SEARCH_QUERY);   // a cold pass
    PairState r;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r, st_dev.p, sizeof(r), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "evaluation pass");
    for (int i = 0; i < 48; ++i) out[i] = r.eval_out[i];
    if (r.nn_overflow) return fail(FRICP_EOVERFLOW, "closest-point search stack overflow");
    if (r.status == FRICP_EDEGENERATE) return fail(FRICP_EDEGENERATE, "degenerate alignment problem");
    return FRICP_OK;
}

}  // extern "C"
