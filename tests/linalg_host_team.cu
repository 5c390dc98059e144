// Host build of the solver's small-algebra routines run by a team of host
// threads (one thread per lane, a barrier for the team's sync), exported with C
// linkage so a CPU test can check that any team size gives the bits of a team
// of one lane: the lane split and the scratch exchange must not change a single
// operation. Packing and scratch offsets are those of tests/linalg_device.cu.
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#define FRICP_HOST_TEAM 1
#include "../paper_2007_07627_gb300/csrc/linalg.cuh"

namespace {
// A barrier whose wait gives up after two seconds (lanes that diverged into
// different numbers of syncs) and records it, so a broken team fails the test
// instead of hanging it.
struct Barrier {
    std::mutex mu;
    std::condition_variable cv;
    int size = 1, waiting = 0, failed = 0;
    unsigned long gen = 0;
    void wait() {
        std::unique_lock<std::mutex> lk(mu);
        if (failed) return;
        const unsigned long g = gen;
        if (++waiting == size) {
            waiting = 0;
            ++gen;
            cv.notify_all();
        } else if (!cv.wait_for(lk, std::chrono::seconds(2), [&] { return gen != g || failed; })) {
            failed = 1;
            cv.notify_all();
        }
    }
};
Barrier g_bar;
thread_local int t_lane = 0;
}  // namespace

namespace fricp {
int fricp_host_team_lane() { return t_lane; }
int fricp_host_team_size() { return g_bar.size; }
void fricp_host_team_sync() { g_bar.wait(); }
}  // namespace fricp

namespace {
using namespace fricp;

void run_case(int op, const double *x, double *y, double *sh) {
    const Team tm{sh};
    const int lane = tm.lane();
    if (op == 0) {
        const int mk = (int)x[0];
        if (lane == 0)
            for (int i = 0; i < 6; ++i) {
                sh[6 * kMaxM + i] = x[1 + 6 * mk + i];
                for (int j = 0; j < mk; ++j) sh[6 * j + i] = x[1 + i * mk + j];
            }
        tm.sync();
        double th[kMaxM];
        const bool ok = anderson_lstsq(tm, sh, mk, th, sh + 48);
        if (lane == 0) {
            y[0] = ok ? 1.0 : 0.0;
            for (int j = 0; j < mk; ++j) y[1 + j] = ok ? th[j] : 0.0;
        }
    } else if (op == 1) {
        if (lane == 0)
            for (int i = 0; i < 42; ++i) sh[i] = x[i];
        tm.sync();
        double v[6];
        const bool ok = chol6_solve(tm, sh, sh + 36, v, sh + 48);
        if (lane == 0) {
            y[0] = ok ? 1.0 : 0.0;
            for (int i = 0; i < 6; ++i) y[1 + i] = ok ? v[i] : 0.0;
        }
    } else if (op == 2) {
        if (lane == 0)
            for (int i = 0; i < 9; ++i) sh[i] = x[i];
        tm.sync();
        const bool ok = procrustes_rotation(tm, sh, sh + 16, sh + 32);
        if (lane == 0) {
            y[0] = ok ? 1.0 : 0.0;
            for (int i = 0; i < 9; ++i) y[1 + i] = ok ? sh[16 + i] : 0.0;
        }
    } else if (op == 3) {
        double xi[6];
        for (int i = 0; i < 6; ++i) xi[i] = x[i];
        se3_exp(tm, xi, sh, sh + 16);
        if (lane == 0)
            for (int i = 0; i < 12; ++i) y[i] = sh[i];
    } else if (op == 4) {
        if (lane == 0)
            for (int i = 0; i < 12; ++i) sh[i] = x[i];
        tm.sync();
        double xi[6];
        se3_log(tm, sh, xi, sh + 16);
        if (lane == 0)
            for (int i = 0; i < 6; ++i) y[i] = xi[i];
    } else if (op == 5) {
        double xi[6];
        for (int i = 0; i < 6; ++i) xi[i] = x[i];
        p2pl_chain(tm, xi, sh, sh + 40);
        if (lane == 0)
            for (int i = 0; i < 36; ++i) y[i] = sh[i];
    }
    tm.sync();   // the scratch is reused by the next case
}
}  // namespace

// n cases of op, each run by a team of `lanes` host threads. in: n * is doubles,
// out: n * os doubles (zeroed first). Returns 0, or 1 if a sync gave up.
extern "C" int t_team_run(int op, int lanes, int n, const double *in, int is, double *out, int os) {
    std::vector<double> sh(kTeamScratch, 0.0);
    for (int k = 0; k < n * os; ++k) out[k] = 0.0;
    g_bar.size = lanes;
    g_bar.waiting = 0;
    g_bar.failed = 0;
    std::vector<std::thread> th;
    for (int l = 0; l < lanes; ++l)
        th.emplace_back([&, l] {
            t_lane = l;
            for (int c = 0; c < n; ++c) run_case(op, in + (size_t)c * is, out + (size_t)c * os, sh.data());
        });
    for (auto &t : th) t.join();
    return g_bar.failed;
}
