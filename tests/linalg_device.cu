// Device build of the solver's small-algebra routines, run by a team of 32
// lanes (one warp per case), exported with C linkage so the GPU tests can
// compare each routine with its host build (a team of one lane) on the same
// inputs. Input and output packing per op (doubles per case):
//   0 anderson_lstsq  in: mk, D (6 x mk, row-major), f (6)   out: ok, theta (mk)
//   1 chol6_solve     in: A (36, row-major), b (6)          out: ok, x (6)
//   2 procrustes      in: H (9)                             out: ok, R (9)
//   3 se3_exp         in: xi (6)                            out: T (12)
//   4 se3_log         in: T (12)                            out: xi (6)
//   5 p2pl_chain      in: xi (6)                            out: K (36)
// The scratch offsets are those of tests/linalg_host.cu.
#include <cuda_runtime.h>

#include "../paper_2007_07627_gb300/csrc/linalg.cuh"

namespace {
using namespace fricp;

__global__ void __launch_bounds__(32) k_team(int op, int n, const double *in, int is, double *out, int os) {
    __shared__ double sh[kTeamScratch];
    const int c = blockIdx.x;
    if (c >= n || threadIdx.x >= kTeamLanes) return;
    const Team tm{sh};
    const double *x = in + (size_t)c * is;
    double *y = out + (size_t)c * os;
    const int lane = tm.lane();
    if (op == 0) {
        const int mk = (int)x[0];
        if (lane == 0) {
            for (int i = 0; i < 6; ++i) {
                sh[6 * kMaxM + i] = x[1 + 6 * mk + i];
                for (int j = 0; j < mk; ++j) sh[6 * j + i] = x[1 + i * mk + j];
            }
        }
        tm.sync();
        double th[kMaxM];
        const bool ok = anderson_lstsq(tm, sh, mk, th, sh + 48);
        if (lane == 0) {
            y[0] = ok ? 1.0 : 0.0;
            for (int j = 0; j < mk; ++j) y[1 + j] = th[j];
        }
    } else if (op == 1) {
        if (lane == 0)
            for (int i = 0; i < 42; ++i) sh[i] = x[i];
        tm.sync();
        double v[6];
        const bool ok = chol6_solve(tm, sh, sh + 36, v, sh + 48);
        if (lane == 0) {
            y[0] = ok ? 1.0 : 0.0;
            for (int i = 0; i < 6; ++i) y[1 + i] = v[i];
        }
    } else if (op == 2) {
        if (lane == 0)
            for (int i = 0; i < 9; ++i) sh[i] = x[i];
        tm.sync();
        const bool ok = procrustes_rotation(tm, sh, sh + 16, sh + 32);
        if (lane == 0) {
            y[0] = ok ? 1.0 : 0.0;
            for (int i = 0; i < 9; ++i) y[1 + i] = sh[16 + i];
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
}
}  // namespace

extern "C" int d_team_run(int op, int n, const double *in_h, int is, double *out_h, int os) {
    double *din = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&din, sizeof(double) * (size_t)n * is);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * (size_t)n * os);
    if (e == cudaSuccess) e = cudaMemcpy(din, in_h, sizeof(double) * (size_t)n * is, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dout, 0, sizeof(double) * (size_t)n * os);
    if (e == cudaSuccess) {
        k_team<<<n, 32>>>(op, n, din, is, dout, os);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out_h, dout, sizeof(double) * (size_t)n * os, cudaMemcpyDeviceToHost);
    if (din) cudaFree(din);
    if (dout) cudaFree(dout);
    return (int)e;
}
