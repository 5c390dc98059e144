// FP64 small dense algebra of the solver step: weighted Procrustes rotation,
// exp/log on SE(3), the Anderson least-squares problem, the App. D chain matrix
// and the 6x6 point-to-plane Gauss-Newton system.
//
// GB300 has few FP64 units: one FP64 warp instruction occupies them for ~64
// cycles whether one lane or all 32 are active. So these routines run on a
// Team, the 32 lanes of one warp: every lane runs the same control flow on the
// same values (the scalar parts cost no more on 32 lanes than on one), and each
// step with independent outputs (the entries of a 3x3 or 6x6 product, the
// columns of a Householder update, the rows of a triangular update) hands one
// output to each lane, exchanged through the team's scratch (shared memory).
// The arithmetic of an output does not depend on which lane computes it, so on
// the host a Team of one lane runs the same code serially with the same results
// (the CPU tests), up to the math library's sin/cos/atan2.
//
// Matrices a lane-parallel step reads live in team scratch (a runtime index
// into a register array would spill to local memory). Every routine syncs the
// team before its first scratch write and after its last.
#pragma once

#include <math.h>
#include <string.h>

#include "fricp_internal.cuh"

namespace fricp {

// Lanes of a device team: the first kTeamLanes lanes of a warp.
#ifndef FRICP_TEAM_LANES
#define FRICP_TEAM_LANES 32
#endif
constexpr int kTeamLanes = FRICP_TEAM_LANES;
constexpr unsigned kTeamMask = kTeamLanes == 32 ? 0xffffffffu : ((1u << kTeamLanes) - 1u);

// A host build that defines FRICP_HOST_TEAM (a CPU test) supplies the three
// functions below and runs a team as host threads; every other host build is a
// team of one lane.
#if !defined(__CUDA_ARCH__) && defined(FRICP_HOST_TEAM)
int fricp_host_team_lane();
int fricp_host_team_size();
void fricp_host_team_sync();
#endif

struct Team {
    double *sh;   // scratch shared by the team: kTeamScratch doubles
    FRICP_HD int lane() const {
#if defined(__CUDA_ARCH__)
        return threadIdx.x & 31;
#elif defined(FRICP_HOST_TEAM)
        return fricp_host_team_lane();
#else
        return 0;
#endif
    }
    FRICP_HD int size() const {
#if defined(__CUDA_ARCH__)
        return kTeamLanes;
#elif defined(FRICP_HOST_TEAM)
        return fricp_host_team_size();
#else
        return 1;
#endif
    }
    FRICP_HD void sync() const {
#if defined(__CUDA_ARCH__)
        __syncwarp(kTeamMask);
#elif defined(FRICP_HOST_TEAM)
        fricp_host_team_sync();
#endif
    }
};

constexpr int kTeamScratch = 512;   // doubles of scratch a solver step needs

// Uniform register array -> scratch (entry e written by lane e mod size).
template <int N>
FRICP_HD inline void t_store(const Team &tm, double *dst, const double *v) {
    const int l = tm.lane(), s = tm.size();
#pragma unroll
    for (int e = 0; e < N; ++e)
        if (e % s == l) dst[e] = v[e];
}

template <int N>
FRICP_HD inline void t_load(const double *src, double (&v)[N]) {
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = src[e];
}

FRICP_HD inline unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

FRICP_HD inline double bitsd(unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// x == +-0 by its bits (integer instructions, not the FP64 pipe)
FRICP_HD inline bool is_zero_bits(double x) { return (dbits(x) << 1) == 0ull; }

FRICP_HD inline void hat3(const double a[3], double H[9]) {
    H[0] = 0.0;   H[1] = -a[2]; H[2] = a[1];
    H[3] = a[2];  H[4] = 0.0;   H[5] = -a[0];
    H[6] = -a[1]; H[7] = a[0];  H[8] = 0.0;
}

FRICP_HD inline void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = fma(a[1], b[2], -(a[2] * b[1]));
    c[1] = fma(a[2], b[0], -(a[0] * b[2]));
    c[2] = fma(a[0], b[1], -(a[1] * b[0]));
}

FRICP_HD inline void mul33(const double A[9], const double B[9], double C[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = fma(A[3 * r + 2], B[6 + c], fma(A[3 * r + 1], B[3 + c], A[3 * r] * B[c]));
}

// C = A B for 3x3 row-major matrices in scratch, one entry per lane; C apart from A and B.
FRICP_HD inline void t_mul33(const Team &tm, const double *A, const double *B, double *C) {
    tm.sync();
    for (int e = tm.lane(); e < 9; e += tm.size()) {
        const int r = e / 3, c = e - 3 * r;
        C[e] = fma(A[3 * r + 2], B[6 + c], fma(A[3 * r + 1], B[3 + c], A[3 * r] * B[c]));
    }
    tm.sync();
}

// Reciprocal and inverse square root from a float seed refined by two Newton
// steps in FP64 (relative error ~1e-16): much shorter dependency chains than
// the IEEE FP64 divide / square root on a GPU with few FP64 units. Arguments
// outside the float range fall back to the IEEE operations. The steps are
// written with explicit fma, so the host build rounds exactly as the device.
FRICP_HD inline double rcp64(double a) {
    const double fa = fabs(a);
    if (!(fa > 1e-30 && fa < 1e30)) return 1.0 / a;
    double y = (double)(1.0f / (float)a);
    y = fma(y, fma(-a, y, 1.0), y);
    y = fma(y, fma(-a, y, 1.0), y);
    return y;
}

FRICP_HD inline double rsqrt64(double a) {
    if (!(a > 1e-30 && a < 1e30)) return 1.0 / sqrt(a);
    double y = (double)(1.0f / sqrtf((float)a));
    y = y * fma(-0.5, (a * y) * y, 1.5);
    y = y * fma(-0.5, (a * y) * y, 1.5);
    return y;
}

// Coefficients of the SO(3)/SE(3) exponential for |w| = th:
// a = sin th / th, b = (1 - cos th) / th^2, c = (th - sin th) / th^3,
// by their Taylor series below th = 1e-2 (truncation < 1e-21).
FRICP_HD inline void exp_coeffs(double th2, double *a, double *b, double *c) {
    if (th2 < 1e-4) {
        *a = 1.0 - th2 * (1.0 / 6.0) * (1.0 - th2 * (1.0 / 20.0) * (1.0 - th2 * (1.0 / 42.0)));
        *b = 0.5 * (1.0 - th2 * (1.0 / 12.0) * (1.0 - th2 * (1.0 / 30.0) * (1.0 - th2 * (1.0 / 56.0))));
        *c = (1.0 / 6.0) * (1.0 - th2 * (1.0 / 20.0) * (1.0 - th2 * (1.0 / 42.0) * (1.0 - th2 * (1.0 / 72.0))));
    } else {
        const double ith = rsqrt64(th2);
        const double th = th2 * ith;
        double sn, cs;
        sincos(th, &sn, &cs);
        *a = sn * ith;
        *b = (1.0 - cs) * ith * ith;
        *c = (th - sn) * ith * ith * ith;
    }
}

// Eq. (9): T = exp([[w^, u], [0, 0]]) in closed form: R = I + a W + b W^2 and
// t = (I + b W + c W^2) u with W = w^. xi = [w; u] uniform; T (R row-major,
// then t) written to scratch. w: 33 doubles of scratch.
FRICP_HD inline void se3_exp(const Team &tm, const double xi[6], double *T, double *w) {
    double *W = w, *W2 = w + 9, *V = w + 18, *sx = w + 27;
    const double th2 = fma(xi[2], xi[2], fma(xi[1], xi[1], xi[0] * xi[0]));
    double a, b, c;
    exp_coeffs(th2, &a, &b, &c);
    double Wr[9];
    hat3(xi, Wr);
    tm.sync();
    t_store<9>(tm, W, Wr);
    t_store<6>(tm, sx, xi);
    t_mul33(tm, W, W, W2);
    for (int e = tm.lane(); e < 9; e += tm.size()) {
        const double I = (e % 4 == 0) ? 1.0 : 0.0;
        T[e] = fma(b, W2[e], fma(a, W[e], I));
        V[e] = fma(c, W2[e], fma(b, W[e], I));
    }
    tm.sync();
    for (int r = tm.lane(); r < 3; r += tm.size())
        T[9 + r] = fma(V[3 * r + 2], sx[5], fma(V[3 * r + 1], sx[4], V[3 * r] * sx[3]));
    tm.sync();
}

// App. A for d = 3: the rotation block has one angle th in [0, pi] and axis k;
// log T = [[th k^, V t], [0, 0]] with V = I - th/2 K + (1 - th sin th / (2 (1 - cos th))) K^2,
// K = k^ (the unit generator), i.e. V = I - W/2 + e W^2 with W = th K and
// e = (1 - th sin th / (2 (1 - cos th))) / th^2 (series below th = 1e-2).
// At th within 1e-3 of pi the axis comes from the symmetric part of R, the
// largest diagonal first, oriented along vee(R - R^T) (the largest-magnitude
// component positive when that vanishes).
// T (12) in scratch; xi uniform. w: 30 doubles of scratch.
FRICP_HD inline void se3_log(const Team &tm, const double *T, double xi[6], double *w) {
    double R[9];
    t_load(T, R);
    const double v0 = 0.5 * (R[7] - R[5]), v1 = 0.5 * (R[2] - R[6]), v2 = 0.5 * (R[3] - R[1]);
    const double sn2 = fma(v2, v2, fma(v1, v1, v0 * v0));
    const double isn = sn2 > 0.0 ? rsqrt64(sn2) : 0.0;   // 1 / sin th (unused when sin th = 0)
    const double sn = sn2 * isn;
    const double cs = 0.5 * (R[0] + R[4] + R[8] - 1.0);
    const double th = atan2(sn, cs);
    const double th2 = th * th;
    double wv[3];
    if (th < 1e-2) {
        // th / sin th = 1 + th^2/6 + 7 th^4/360 + 31 th^6/15120
        const double f = 1.0 + th2 * (1.0 / 6.0) + th2 * th2 * (7.0 / 360.0) + th2 * th2 * th2 * (31.0 / 15120.0);
        wv[0] = f * v0; wv[1] = f * v1; wv[2] = f * v2;
    } else if (3.141592653589793 - th < 1e-3) {
        const double omc = 1.0 - cs;
        double S[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                S[3 * r + c] = (0.5 * (R[3 * r + c] + R[3 * c + r]) - (r == c ? cs : 0.0)) / omc;
        const int i = (S[4] > S[0]) ? (S[8] > S[4] ? 2 : 1) : (S[8] > S[0] ? 2 : 0);
        const double Si[3] = {S[3 * i], S[3 * i + 1], S[3 * i + 2]};
        const double ki = sqrt(fmax(i == 0 ? Si[0] : (i == 1 ? Si[1] : Si[2]), 0.0));
        double k[3];
        for (int j = 0; j < 3; ++j) k[j] = (j == i) ? ki : Si[j] / ki;
        double dir = k[0] * v0 + k[1] * v1 + k[2] * v2;
        if (dir == 0.0) {
            double big = k[0];
            if (fabs(k[1]) > fabs(big)) big = k[1];
            if (fabs(k[2]) > fabs(big)) big = k[2];
            dir = big;
        }
        const double sg = dir < 0.0 ? -1.0 : 1.0;
        const double nk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        for (int j = 0; j < 3; ++j) wv[j] = sg * th * k[j] / nk;
    } else {
        const double f = th * isn;
        wv[0] = f * v0; wv[1] = f * v1; wv[2] = f * v2;
    }
    double e;
    if (th < 1e-2) {
        e = 1.0 / 12.0 + th2 * (1.0 / 720.0) + th2 * th2 * (1.0 / 30240.0);
    } else {
        // sin th and cos th are sn and cs themselves (R orthogonal): no sincos
        const double omc2 = 2.0 * (1.0 - cs);
        e = (omc2 - th * sn) * rcp64(omc2 * th2);
    }
    double *W = w, *W2 = w + 9, *V = w + 18, *u = w + 27;
    double Wr[9];
    hat3(wv, Wr);
    tm.sync();
    t_store<9>(tm, W, Wr);
    t_mul33(tm, W, W, W2);
    for (int i = tm.lane(); i < 9; i += tm.size())
        V[i] = fma(e, W2[i], fma(-0.5, W[i], (i % 4 == 0) ? 1.0 : 0.0));
    tm.sync();
    for (int r = tm.lane(); r < 3; r += tm.size())
        u[r] = fma(V[3 * r + 2], T[11], fma(V[3 * r + 1], T[10], V[3 * r] * T[9]));
    tm.sync();
    xi[0] = wv[0]; xi[1] = wv[1]; xi[2] = wv[2];
    xi[3] = u[0]; xi[4] = u[1]; xi[5] = u[2];
}

// Rotation of the weighted Procrustes problem (Eq. 4 / Eq. 12, "closed form via
// SVD"): R maximises tr(R H) over SO(3) for H = sum w (p - pbar)(q - qbar)^T,
// i.e. R = V diag(1,1,d) U^T with H = U S V^T and d = sign det(V U^T).
//
// Computed in three parts:
//   1. a one-sided (Hestenes) Jacobi SVD of H / max|H| in float; the singular
//      vector of the smallest singular value is completed by a cross product,
//      so a rank-2 H (planar data) keeps a unique answer; R0 = V diag(1,1,d) U^T;
//   2. two Newton-Schulz steps R <- R (3 I - R^T R) / 2 in FP64 make R0
//      orthogonal to FP64 precision;
//   3. two Newton steps on SO(3) in FP64: with A = R H, g = vee(A - A^T) and
//      K = tr(A) I - (A + A^T) / 2 (positive definite near the maximiser),
//      w = K^-1 g and R <- exp(w^) R. Each step squares the float error, so
//      R is the FP64 maximiser (the same one the FP64 SVD gives).
// H (9) and R (9) in scratch. Returns false when rank(H) < 2 or the Newton
// system is not positive definite. w: 60 doubles of scratch.
FRICP_HD inline bool procrustes_rotation(const Team &tm, const double *H, double *R, double *w) {
    double *N = w, *Tm = w + 9, *Am = w + 18, *W = w + 27, *W2 = w + 36, *E = w + 45;
    float *Af = reinterpret_cast<float *>(w + 54);   // 9 floats
    unsigned long long mx = 0ull;   // max |H| on the bits (nonnegative doubles order as integers)
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const unsigned long long b = dbits(H[i]) & 0x7fffffffffffffffull;
        mx = b > mx ? b : mx;
    }
    if (mx == 0ull || mx >= 0x7ff0000000000000ull) return false;   // zero, or an inf / NaN entry
    const double ihm = rcp64(bitsd(mx));
    tm.sync();
    for (int e = tm.lane(); e < 9; e += tm.size()) Af[e] = (float)(H[e] * ihm);
    tm.sync();
    float A[9], V[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        A[i] = Af[i];
        V[i] = (i % 4 == 0) ? 1.0f : 0.0f;
    }
    for (int sweep = 0; sweep < 12; ++sweep) {
        float off = 0.0f;
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {   // column pairs (0,1), (0,2), (1,2)
            const int p = pr == 2 ? 1 : 0, q = pr == 0 ? 1 : 2;
            float al = 0.0f, be = 0.0f, ga = 0.0f;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                al = fmaf(A[3 * r + p], A[3 * r + p], al);
                be = fmaf(A[3 * r + q], A[3 * r + q], be);
                ga = fmaf(A[3 * r + p], A[3 * r + q], ga);
            }
            if (ga == 0.0f) continue;
            const float rel = fabsf(ga) / sqrtf(al * be);
            off = fmaxf(off, rel);
            if (!(rel > 1e-8f)) continue;
            const float zeta = (be - al) / (2.0f * ga);
            const float t = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
            const float cs = 1.0f / sqrtf(1.0f + t * t), sn = cs * t;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float ap = A[3 * r + p], aq = A[3 * r + q];
                A[3 * r + p] = cs * ap - sn * aq;
                A[3 * r + q] = sn * ap + cs * aq;
                const float vp = V[3 * r + p], vq = V[3 * r + q];
                V[3 * r + p] = cs * vp - sn * vq;
                V[3 * r + q] = sn * vp + cs * vq;
            }
        }
        if (off <= 1e-7f) break;
    }
    // completion (every index a compile-time constant; the column roles are selects)
    float sg[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) sg[j] = sqrtf(A[j] * A[j] + A[3 + j] * A[3 + j] + A[6 + j] * A[6 + j]);
    int kmin = 0;
    if (sg[1] < sg[0]) kmin = 1;
    if (sg[2] < (kmin == 1 ? sg[1] : sg[0])) kmin = 2;
    const bool a0 = kmin != 0;   // column a: 0 unless kmin == 0 (then 1)
    const bool b1 = kmin == 2;   // column b: 2 unless kmin == 2 (then 1)
    const float sa = a0 ? sg[0] : sg[1], sb = b1 ? sg[1] : sg[2];
    const float smax = fmaxf(sa, sb), smid = fminf(sa, sb);
    if (!(smid > 1e-6f * smax) || !(smax > 0.0f)) return false;
    float U[9], ua[3], ub[3], uk[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        ua[r] = (a0 ? A[3 * r] : A[3 * r + 1]) / sa;
        ub[r] = (b1 ? A[3 * r + 1] : A[3 * r + 2]) / sb;
    }
    uk[0] = ua[1] * ub[2] - ua[2] * ub[1];
    uk[1] = ua[2] * ub[0] - ua[0] * ub[2];
    uk[2] = ua[0] * ub[1] - ua[1] * ub[0];
    const float nk = 1.0f / sqrtf(uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool is_a = (c == 0 && a0) || (c == 1 && !a0);
            U[3 * r + c] = c == kmin ? uk[r] * nk : (is_a ? ua[r] : ub[r]);
        }
    }
    const float detV = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                       V[2] * (V[3] * V[7] - V[4] * V[6]);
    const float detU = U[0] * (U[4] * U[8] - U[5] * U[7]) - U[1] * (U[3] * U[8] - U[5] * U[6]) +
                       U[2] * (U[3] * U[7] - U[4] * U[6]);
    const float d = (detV * detU) < 0.0f ? -1.0f : 1.0f;
    float R0[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 3; ++j) acc += V[3 * r + j] * (j == kmin ? d : 1.0f) * U[3 * c + j];
            R0[3 * r + c] = acc;
        }
    {   // each lane widens its own entry (one FP64 conversion per lane)
        const int l = tm.lane();
        for (int e = l; e < 9; e += tm.size()) {
            float mine = R0[0];
#pragma unroll
            for (int k = 1; k < 9; ++k) mine = (e == k) ? R0[k] : mine;
            R[e] = (double)mine;
        }
    }
    tm.sync();
    // Newton-Schulz: orthogonal to FP64 precision
    for (int it = 0; it < 2; ++it) {
        for (int e = tm.lane(); e < 9; e += tm.size()) {
            const int r = e / 3, c = e - 3 * r;
            const double m = fma(R[6 + r], R[6 + c], fma(R[3 + r], R[3 + c], R[r] * R[c]));
            N[e] = fma(-0.5, m, (e % 4 == 0) ? 1.5 : 0.0);
        }
        t_mul33(tm, R, N, Tm);
        for (int e = tm.lane(); e < 9; e += tm.size()) R[e] = Tm[e];
        tm.sync();
    }
    // Newton on SO(3): R <- exp(w^) R with (tr(A) I - sym(A)) w = vee(A - A^T), A = R H
    for (int it = 0; it < 2; ++it) {
        t_mul33(tm, R, H, Am);
        double a[9];
        t_load(Am, a);
        const double g[3] = {a[5] - a[7], a[6] - a[2], a[1] - a[3]};
        const double tr = a[0] + a[4] + a[8];
        const double k00 = tr - a[0], k11 = tr - a[4], k22 = tr - a[8];
        const double k01 = -0.5 * (a[1] + a[3]), k02 = -0.5 * (a[2] + a[6]), k12 = -0.5 * (a[5] + a[7]);
        const double c00 = fma(k11, k22, -(k12 * k12)), c01 = fma(k02, k12, -(k01 * k22));
        const double c02 = fma(k01, k12, -(k02 * k11)), c11 = fma(k00, k22, -(k02 * k02));
        const double c12 = fma(k01, k02, -(k00 * k12)), c22 = fma(k00, k11, -(k01 * k01));
        const double det = fma(k02, c02, fma(k01, c01, k00 * c00));
        if (!(det > 0.0) || !(k00 > 0.0) || !isfinite(det)) return false;
        const double idet = rcp64(det);
        const double wv[3] = {fma(c02, g[2], fma(c01, g[1], c00 * g[0])) * idet,
                              fma(c12, g[2], fma(c11, g[1], c01 * g[0])) * idet,
                              fma(c22, g[2], fma(c12, g[1], c02 * g[0])) * idet};
        double ea, eb, ec;
        exp_coeffs(fma(wv[2], wv[2], fma(wv[1], wv[1], wv[0] * wv[0])), &ea, &eb, &ec);
        double Wr[9];
        hat3(wv, Wr);
        t_store<9>(tm, W, Wr);
        t_mul33(tm, W, W, W2);
        for (int e = tm.lane(); e < 9; e += tm.size()) E[e] = fma(eb, W2[e], fma(ea, W[e], (e % 4 == 0) ? 1.0 : 0.0));
        t_mul33(tm, E, R, Tm);
        for (int e = tm.lane(); e < 9; e += tm.size()) R[e] = Tm[e];
        tm.sync();
    }
    return true;
}

// Six-term dot product as a balanced tree (short dependency chain).
FRICP_HD inline double dot6(const double a[6], const double b[6]) {
    const double s01 = fma(a[1], b[1], a[0] * b[0]);
    const double s23 = fma(a[3], b[3], a[2] * b[2]);
    const double s45 = fma(a[5], b[5], a[4] * b[4]);
    return (s01 + s23) + s45;
}

// Anderson coefficients (Sec. 4.1, Eq. 6): theta = argmin || f - D theta ||_2 for
// a 6 x mk matrix D, by Householder QR. Dm holds the columns of D (column c at
// Dm + 6 c, c < mk) and f at Dm + 6 kMaxM, in scratch; both are overwritten.
// Each reflector is formed by every lane; the columns it updates are split over
// the lanes. Returns false under the rank rule (min |R_jj| < 1e-14 max |R_jj|)
// or a non-finite theta. w: 8 doubles of scratch.
FRICP_HD inline bool anderson_lstsq(const Team &tm, double *Dm, int mk, double theta[kMaxM], double *w) {
    double Rd[kMaxM];
#pragma unroll
    for (int j = 0; j < kMaxM; ++j) {
        Rd[j] = 0.0;
        if (j >= mk) continue;
        double v[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] = (i < j) ? 0.0 : Dm[6 * j + i];
        const double nrm2 = dot6(v, v);
        const double nrm = nrm2 > 0.0 ? nrm2 * rsqrt64(nrm2) : 0.0;
        const double alpha = -copysign(nrm, v[j]);
        Rd[j] = alpha;
        if (nrm == 0.0) continue;
        // v = x - alpha e_j has |v_j| = |x_j| + nrm, so v.v = 2 (nrm^2 + |x_j| nrm)
        const double vv2 = fma(fabs(v[j]), nrm, nrm2);
        v[j] -= alpha;
        const double ivv2 = rcp64(vv2);   // 2 / v.v
        tm.sync();   // every lane has read column j
        for (int c = j + 1 + tm.lane(); c <= kMaxM; c += tm.size()) {
            if (c >= mk && c != kMaxM) continue;
            double *col = Dm + 6 * c;
            double x[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) x[i] = (i < j) ? 0.0 : col[i];
            const double sc = dot6(v, x) * ivv2;
#pragma unroll
            for (int i = j; i < 6; ++i) col[i] = fma(-sc, v[i], col[i]);
        }
        tm.sync();
    }
    double rmax = 0.0, rmin = INFINITY;
#pragma unroll
    for (int j = 0; j < kMaxM; ++j) {
        if (j >= mk) continue;
        rmax = fmax(rmax, fabs(Rd[j]));
        rmin = fmin(rmin, fabs(Rd[j]));
    }
    if (!isfinite(rmax) || rmax == 0.0 || rmin < 1e-14 * rmax) return false;
    // 1 / R_jj, one per lane
    for (int j = tm.lane(); j < mk; j += tm.size()) {
        double rj = Rd[0];
#pragma unroll
        for (int k = 1; k < kMaxM; ++k) rj = (j == k) ? Rd[k] : rj;
        w[j] = rcp64(rj);
    }
    tm.sync();
    const double *f = Dm + 6 * kMaxM;
#pragma unroll
    for (int j = kMaxM - 1; j >= 0; --j) {
        theta[j] = 0.0;
        if (j >= mk) continue;
        double acc = f[j];
#pragma unroll
        for (int c = j + 1; c < kMaxM; ++c)
            if (c < mk) acc = fma(-Dm[6 * c + j], theta[c], acc);
        theta[j] = acc * w[j];
        if (!isfinite(theta[j])) return false;
    }
    return true;
}

// Cholesky solve of a 6x6 symmetric positive-definite system; false if a pivot
// is not positive and finite. A (row-major; its lower triangle and diagonal are
// read) and b in scratch, x uniform. A direction whose row, column and
// right-hand side are all exactly zero gets x_j = 0: the system of points in a
// plane (z = 0, in-plane normals), where tilting the plane and moving along z
// change no distance, is the 2-D system (Sec. 3 states the problem in R^d).
// Such a direction is solved as the decoupled row 1 * x_j = 0, which leaves
// every other entry of the factor bit-identical to the factor without it.
// 3-D data never has such a direction, and then nothing changes.
// Right-looking (outer-product) elimination: at column j every lane updates its
// own entries of the trailing triangle. w: 48 doubles of scratch.
FRICP_HD inline bool chol6_solve(const Team &tm, const double *A, const double *b, double x[6], double *w) {
    double *L = w, *y = w + 36;
    bool zero[6];
    int na = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        bool z = is_zero_bits(b[j]) && is_zero_bits(A[7 * j]);   // a zero row has a zero diagonal: test that first
        for (int k = 0; k < 6 && z; ++k) z = is_zero_bits(k < j ? A[6 * j + k] : A[6 * k + j]);
        zero[j] = z;
        na += z ? 0 : 1;
        x[j] = 0.0;
    }
    if (na == 0) return false;
    tm.sync();
    for (int e = tm.lane(); e < 36; e += tm.size()) {
        const int r = e / 6, c = e - 6 * r;
        L[e] = (r >= c) ? A[e] : 0.0;
    }
    for (int e = tm.lane(); e < 6; e += tm.size()) y[e] = b[e];
    tm.sync();
    for (int e = tm.lane(); e < 6; e += tm.size()) {
        bool z = false;
#pragma unroll
        for (int k = 0; k < 6; ++k) z = (e == k) ? zero[k] : z;
        if (z) L[7 * e] = 1.0;
    }
    tm.sync();
    double il[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const double d = L[7 * j];
        if (!(d > 0.0) || !isfinite(d)) return false;
        il[j] = rsqrt64(d);   // 1 / L_jj
        tm.sync();
        for (int i = j + 1 + tm.lane(); i < 6; i += tm.size()) L[6 * i + j] *= il[j];
        tm.sync();
        // trailing update L_ik -= L_ij L_kj for j < k <= i, one entry per lane
        const int nt = (5 - j) * (6 - j) / 2;
        for (int p = tm.lane(); p < nt; p += tm.size()) {
            int i = j + 1, q = p;
            while (q > i - j - 1) {
                q -= i - j;
                ++i;
            }
            const int k = j + 1 + q;
            L[6 * i + k] = fma(-L[6 * i + j], L[6 * k + j], L[6 * i + k]);
        }
        tm.sync();
    }
    // forward: L y = b (column by column: the same operation order as row sums)
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double yi = y[i] * il[i];
        tm.sync();
        for (int k = i + 1 + tm.lane(); k < 6; k += tm.size()) y[k] = fma(-L[6 * k + i], yi, y[k]);
        if (tm.lane() == 0) y[i] = yi;
        tm.sync();
    }
    // backward: L^T x = y
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        const double xi = y[i] * il[i];
        tm.sync();
        for (int k = tm.lane(); k < i; k += tm.size()) y[k] = fma(-L[6 * i + k], xi, y[k]);
        tm.sync();
        x[i] = xi;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j)
        if (zero[j]) x[j] = 0.0;
    return true;
}

// Chain matrix K of App. D: the gradient of B_i(xi) = (R p_i + t - q_i) . n_i at
// xi = [delta; u] factors as J_i = K z_i with z_i = [y_i x n_i; n_i], y_i = R p_i,
// because dR/d delta_j = w_j^ R with w_j = (delta_j delta + delta x (I - R) e_j) / |delta|^2
// (so n . (dR/d delta_j) p = w_j . (y x n)). Rows 0..2: [w_j^T, (dt/d delta_j)^T];
// rows 3..5: [0, (dt/du_j)^T], with dt/d delta and dt/du as printed in App. D.
// delta = 0 takes App. D's special case; 0 < |delta| < 1e-6 a second-order series.
// K (36, row-major) written to scratch. w: 123 doubles of scratch.
FRICP_HD inline void p2pl_chain(const Team &tm, const double xi[6], double *K, double *w) {
    const double *d = xi, *u = xi + 3;
    const double th2 = fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0]));
    if (th2 == 0.0 || th2 < 1e-12) {   // the rare near-identity cases, by every lane alike
        double Kr[36];
        for (int i = 0; i < 36; ++i) Kr[i] = 0.0;
        if (th2 == 0.0) {
            for (int j = 0; j < 3; ++j) {
                Kr[6 * j + j] = 1.0;
                Kr[6 * (3 + j) + 3 + j] = 1.0;
            }
        } else {
            double Dh[9], D2[9], Jl[9];
            hat3(d, Dh);
            mul33(Dh, Dh, D2);
            for (int i = 0; i < 9; ++i) Jl[i] = ((i % 4 == 0) ? 1.0 : 0.0) + 0.5 * Dh[i] + D2[i] / 6.0;
            double du[3];
            cross3(d, u, du);
            for (int j = 0; j < 3; ++j) {
                double e[3] = {0.0, 0.0, 0.0};
                e[j] = 1.0;
                double exu[3], ex_du[3], d_exu[3];
                cross3(e, u, exu);
                cross3(e, du, ex_du);
                cross3(d, exu, d_exu);
                for (int a = 0; a < 3; ++a) {
                    Kr[6 * j + a] = Jl[3 * a + j];                                      // w_j = J_l e_j
                    Kr[6 * j + 3 + a] = 0.5 * exu[a] + (ex_du[a] + d_exu[a]) / 6.0;     // dt/d delta_j
                    Kr[6 * (3 + j) + 3 + a] = Jl[3 * a + j];                            // dt/du_j
                }
            }
        }
        tm.sync();
        t_store<36>(tm, K, Kr);
        tm.sync();
        return;
    }
    double *Tr = w, *ImR = w + 12, *Wm = w + 21, *M = w + 30, *Dh = w + 39, *Uh = w + 48, *C = w + 57;
    double *Dt = w + 66, *v = w + 75, *Md = w + 87, *ew = w + 90;   // v: d, u, u x d, R (u x d); ew: 33
    const double xr[6] = {d[0], d[1], d[2], 0.0, 0.0, 0.0};
    se3_exp(tm, xr, Tr, ew);
    const double ith2 = rcp64(th2);
    const double du_dot = fma(d[2], u[2], fma(d[1], u[1], d[0] * u[0]));
    double Dhr[9], Uhr[9], uxd[3];
    hat3(d, Dhr);
    hat3(u, Uhr);
    cross3(u, d, uxd);
    const double vv[9] = {d[0], d[1], d[2], u[0], u[1], u[2], uxd[0], uxd[1], uxd[2]};
    tm.sync();
    t_store<9>(tm, Dh, Dhr);
    t_store<9>(tm, Uh, Uhr);
    t_store<9>(tm, v, vv);
    for (int e = tm.lane(); e < 9; e += tm.size()) ImR[e] = ((e % 4 == 0) ? 1.0 : 0.0) - Tr[e];
    tm.sync();
    // w_j (row j of Wm) = (d_j d + d x (I - R) e_j) / th^2
    for (int e = tm.lane(); e < 9; e += tm.size()) {
        const int j = e / 3, a = e - 3 * j, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
        const double cr = fma(v[a1], ImR[3 * a2 + j], -(v[a2] * ImR[3 * a1 + j]));
        Wm[e] = fma(v[j], v[a], cr) * ith2;
    }
    // M = (R - I) u^ + (d . u) I
    for (int e = tm.lane(); e < 9; e += tm.size()) {
        const int r = e / 3, c = e - 3 * r;
        const double m = fma(-ImR[3 * r + 2], Uh[6 + c], fma(-ImR[3 * r + 1], Uh[3 + c], -ImR[3 * r] * Uh[c]));
        M[e] = (r == c) ? m + du_dot : m;
    }
    // C = ((I - R) d^ + d d^T) / th^2 (C[3 r + c] = dt_r / du_c)
    for (int e = tm.lane(); e < 9; e += tm.size()) {
        const int r = e / 3, c = e - 3 * r;
        const double m = fma(ImR[3 * r + 2], Dh[6 + c], fma(ImR[3 * r + 1], Dh[3 + c], ImR[3 * r] * Dh[c]));
        C[e] = fma(v[r], v[c], m) * ith2;
    }
    tm.sync();
    // R (u x delta) and M delta
    for (int r = tm.lane(); r < 3; r += tm.size()) {
        v[9 + r] = fma(Tr[3 * r + 2], v[8], fma(Tr[3 * r + 1], v[7], Tr[3 * r] * v[6]));
        Md[r] = fma(M[3 * r + 2], v[2], fma(M[3 * r + 1], v[1], M[3 * r] * v[0]));
    }
    tm.sync();
    // Dt[a][j] = dt_a / d delta_j = (M_aj + d_a u_j + (w_j x R (u x d))_a) / th^2 - 2 (M d)_a d_j / th^4
    for (int e = tm.lane(); e < 9; e += tm.size()) {
        const int a = e / 3, j = e - 3 * a, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
        const double Dj = fma(Wm[3 * j + a1], v[9 + a2], -(Wm[3 * j + a2] * v[9 + a1]));
        Dt[e] = fma((fma(v[a], v[3 + j], M[e]) + Dj), ith2, -(2.0 * ith2 * ith2 * Md[a] * v[j]));
    }
    tm.sync();
    for (int e = tm.lane(); e < 36; e += tm.size()) {
        const int r = e / 6, c = e - 6 * r;
        double k = 0.0;
        if (r < 3)
            k = (c < 3) ? Wm[3 * r + c] : Dt[3 * (c - 3) + r];
        else if (c >= 3)
            k = C[3 * (c - 3) + (r - 3)];
        K[e] = k;
    }
    tm.sync();
}

}  // namespace fricp
