// FP64 small dense algebra run by one thread per registration at the end of
// every fused step: weighted Procrustes rotation, exp/log on SE(3), the Anderson
// least-squares problem and the 6x6 point-to-plane Gauss-Newton system.
#pragma once

#include <math.h>

#include "fricp_internal.cuh"

namespace fricp {

FRICP_HD inline void hat3(const double a[3], double H[9]) {
    H[0] = 0.0;   H[1] = -a[2]; H[2] = a[1];
    H[3] = a[2];  H[4] = 0.0;   H[5] = -a[0];
    H[6] = -a[1]; H[7] = a[0];  H[8] = 0.0;
}

FRICP_HD inline void mul33(const double A[9], const double B[9], double C[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

FRICP_HD inline void mulv3(const double A[9], const double x[3], double y[3]) {
    for (int r = 0; r < 3; ++r) y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}

FRICP_HD inline void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

FRICP_HD inline double det33(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// Reciprocal and inverse square root from a float seed refined by two Newton
// steps in FP64 (relative error ~1e-16): much shorter dependency chains than
// the IEEE FP64 divide / square root on a GPU with few FP64 units. Arguments
// outside the float range fall back to the IEEE operations.
FRICP_HD inline double rcp64(double a) {
    const double fa = fabs(a);
    if (!(fa > 1e-30 && fa < 1e30)) return 1.0 / a;
    double y = (double)(1.0f / (float)a);
    y = y + y * (1.0 - a * y);
    y = y + y * (1.0 - a * y);
    return y;
}

FRICP_HD inline double rsqrt64(double a) {
    if (!(a > 1e-30 && a < 1e30)) return 1.0 / sqrt(a);
    double y = (double)(1.0f / sqrtf((float)a));
    y = y * (1.5 - 0.5 * a * y * y);
    y = y * (1.5 - 0.5 * a * y * y);
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
// t = (I + b W + c W^2) u with W = w^. T: R row-major (9) then t (3).
FRICP_HD inline void se3_exp(const double xi[6], double T[12]) {
    double W[9], W2[9], a, b, c;
    hat3(xi, W);
    mul33(W, W, W2);
    exp_coeffs(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2], &a, &b, &c);
    double V[9];
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        T[i] = I + a * W[i] + b * W2[i];
        V[i] = I + b * W[i] + c * W2[i];
    }
    mulv3(V, xi + 3, T + 9);
}

// App. A for d = 3: the rotation block has one angle th in [0, pi] and axis k;
// log T = [[th k^, V t], [0, 0]] with V = I - th/2 K + (1 - th sin th / (2 (1 - cos th))) K^2,
// K = k^ (the unit generator), i.e. V = I - W/2 + e W^2 with W = th K and
// e = (1 - th sin th / (2 (1 - cos th))) / th^2 (series below th = 1e-2).
// At th within 1e-3 of pi the axis comes from the symmetric part of R, the
// largest diagonal first, oriented along vee(R - R^T) (the largest-magnitude
// component positive when that vanishes).
FRICP_HD inline void se3_log(const double T[12], double xi[6]) {
    const double *R = T;
    const double v0 = 0.5 * (R[7] - R[5]), v1 = 0.5 * (R[2] - R[6]), v2 = 0.5 * (R[3] - R[1]);
    const double sn = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    const double cs = 0.5 * (R[0] + R[4] + R[8] - 1.0);
    const double th = atan2(sn, cs);
    const double th2 = th * th;
    double w[3];
    if (th < 1e-2) {
        // th / sin th = 1 + th^2/6 + 7 th^4/360 + 31 th^6/15120
        const double f = 1.0 + th2 * (1.0 / 6.0) + th2 * th2 * (7.0 / 360.0) + th2 * th2 * th2 * (31.0 / 15120.0);
        w[0] = f * v0; w[1] = f * v1; w[2] = f * v2;
    } else if (3.141592653589793 - th < 1e-3) {
        const double omc = 1.0 - cs;
        double S[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                S[3 * r + c] = (0.5 * (R[3 * r + c] + R[3 * c + r]) - (r == c ? cs : 0.0)) / omc;
        int i = 0;
        if (S[4] > S[0]) i = 1;
        if (S[8] > S[4 * i]) i = 2;
        double k[3];
        k[i] = sqrt(fmax(S[4 * i], 0.0));
        for (int j = 0; j < 3; ++j)
            if (j != i) k[j] = S[3 * i + j] / k[i];
        double dir = k[0] * v0 + k[1] * v1 + k[2] * v2;
        if (dir == 0.0) {
            int big = 0;
            if (fabs(k[1]) > fabs(k[big])) big = 1;
            if (fabs(k[2]) > fabs(k[big])) big = 2;
            dir = k[big];
        }
        const double sg = dir < 0.0 ? -1.0 : 1.0;
        const double nk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        for (int j = 0; j < 3; ++j) w[j] = sg * th * k[j] / nk;
    } else {
        const double f = th * rcp64(sn);
        w[0] = f * v0; w[1] = f * v1; w[2] = f * v2;
    }
    double e;
    if (th < 1e-2) {
        e = 1.0 / 12.0 + th2 * (1.0 / 720.0) + th2 * th2 * (1.0 / 30240.0);
    } else {
        double st, ct;
        sincos(th, &st, &ct);
        e = (1.0 - th * st * rcp64(2.0 * (1.0 - ct))) * rcp64(th2);
    }
    double W[9], W2[9];
    hat3(w, W);
    mul33(W, W, W2);
    double V[9];
    for (int i = 0; i < 9; ++i) V[i] = ((i % 4 == 0) ? 1.0 : 0.0) - 0.5 * W[i] + e * W2[i];
    xi[0] = w[0]; xi[1] = w[1]; xi[2] = w[2];
    mulv3(V, T + 9, xi + 3);
}

// Rotation of the weighted Procrustes problem (Eq. 4 / Eq. 12, "closed form via
// SVD"): R maximises tr(R H) over SO(3) for H = sum w (p - pbar)(q - qbar)^T,
// i.e. R = V diag(1,1,d) U^T with H = U S V^T and d = sign det(V U^T).
//
// Computed in three parts, since dependent FP64 operations are slow on this GPU:
//   1. a one-sided (Hestenes) Jacobi SVD of H / max|H| in float; the singular
//      vector of the smallest singular value is completed by a cross product,
//      so a rank-2 H (planar data) keeps a unique answer; R0 = V diag(1,1,d) U^T;
//   2. two Newton-Schulz steps R <- R (3 I - R^T R) / 2 in FP64 make R0
//      orthogonal to FP64 precision;
//   3. two Newton steps on SO(3) in FP64: with A = R H, g = vee(A - A^T) and
//      K = tr(A) I - (A + A^T) / 2 (positive definite near the maximiser),
//      w = K^-1 g and R <- exp(w^) R. Each step squares the float error, so
//      R is the FP64 maximiser (the same one the FP64 SVD gives).
// Returns false when rank(H) < 2 or the Newton system is not positive definite.
FRICP_HD inline bool procrustes_rotation(const double H[9], double R[9]) {
    double hmax = 0.0;
    for (int i = 0; i < 9; ++i) hmax = fmax(hmax, fabs(H[i]));
    if (!(hmax > 0.0) || !isfinite(hmax)) return false;
    const double ihm = rcp64(hmax);
    float A[9], V[9];
    for (int i = 0; i < 9; ++i) {
        A[i] = (float)(H[i] * ihm);
        V[i] = (i % 4 == 0) ? 1.0f : 0.0f;
    }
    const int P_[3] = {0, 0, 1}, Q_[3] = {1, 2, 2};
    for (int sweep = 0; sweep < 12; ++sweep) {
        float off = 0.0f;
        for (int pr = 0; pr < 3; ++pr) {
            const int p = P_[pr], q = Q_[pr];
            float al = 0.0f, be = 0.0f, ga = 0.0f;
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
    float sg[3];
    for (int j = 0; j < 3; ++j) sg[j] = sqrtf(A[j] * A[j] + A[3 + j] * A[3 + j] + A[6 + j] * A[6 + j]);
    int kmin = 0;
    if (sg[1] < sg[kmin]) kmin = 1;
    if (sg[2] < sg[kmin]) kmin = 2;
    const int a = (kmin == 0) ? 1 : 0;
    const int b = (kmin == 2) ? 1 : 2;
    const float smax = fmaxf(sg[a], sg[b]), smid = fminf(sg[a], sg[b]);
    if (!(smid > 1e-6f * smax) || !(smax > 0.0f)) return false;
    float U[9], ua[3], ub[3], uk[3];
    for (int r = 0; r < 3; ++r) {
        ua[r] = A[3 * r + a] / sg[a];
        ub[r] = A[3 * r + b] / sg[b];
    }
    uk[0] = ua[1] * ub[2] - ua[2] * ub[1];
    uk[1] = ua[2] * ub[0] - ua[0] * ub[2];
    uk[2] = ua[0] * ub[1] - ua[1] * ub[0];
    const float nk = 1.0f / sqrtf(uk[0] * uk[0] + uk[1] * uk[1] + uk[2] * uk[2]);
    for (int r = 0; r < 3; ++r) {
        U[3 * r + a] = ua[r];
        U[3 * r + b] = ub[r];
        U[3 * r + kmin] = uk[r] * nk;
    }
    const float detV = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                       V[2] * (V[3] * V[7] - V[4] * V[6]);
    const float detU = U[0] * (U[4] * U[8] - U[5] * U[7]) - U[1] * (U[3] * U[8] - U[5] * U[6]) +
                       U[2] * (U[3] * U[7] - U[4] * U[6]);
    const float d = (detV * detU) < 0.0f ? -1.0f : 1.0f;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            float acc = 0.0f;
            for (int j = 0; j < 3; ++j) acc += V[3 * r + j] * (j == kmin ? d : 1.0f) * U[3 * c + j];
            R[3 * r + c] = (double)acc;
        }
    // Newton-Schulz: orthogonal to FP64 precision
    for (int it = 0; it < 2; ++it) {
        double RtR[9], T[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                RtR[3 * r + c] = R[r] * R[c] + R[3 + r] * R[3 + c] + R[6 + r] * R[6 + c];
        for (int i = 0; i < 9; ++i) RtR[i] = ((i % 4 == 0) ? 1.5 : 0.0) - 0.5 * RtR[i];
        mul33(R, RtR, T);
        for (int i = 0; i < 9; ++i) R[i] = T[i];
    }
    // Newton on SO(3): R <- exp(w^) R with (tr(A) I - sym(A)) w = vee(A - A^T), A = R H
    for (int it = 0; it < 2; ++it) {
        double Am[9];
        mul33(R, H, Am);
        const double g[3] = {Am[5] - Am[7], Am[6] - Am[2], Am[1] - Am[3]};
        const double tr = Am[0] + Am[4] + Am[8];
        const double k00 = tr - Am[0], k11 = tr - Am[4], k22 = tr - Am[8];
        const double k01 = -0.5 * (Am[1] + Am[3]), k02 = -0.5 * (Am[2] + Am[6]), k12 = -0.5 * (Am[5] + Am[7]);
        const double c00 = k11 * k22 - k12 * k12, c01 = k02 * k12 - k01 * k22, c02 = k01 * k12 - k02 * k11;
        const double c11 = k00 * k22 - k02 * k02, c12 = k01 * k02 - k00 * k12, c22 = k00 * k11 - k01 * k01;
        const double det = k00 * c00 + k01 * c01 + k02 * c02;
        if (!(det > 0.0) || !(k00 > 0.0) || !isfinite(det)) return false;
        const double idet = rcp64(det);
        const double w[3] = {(c00 * g[0] + c01 * g[1] + c02 * g[2]) * idet,
                             (c01 * g[0] + c11 * g[1] + c12 * g[2]) * idet,
                             (c02 * g[0] + c12 * g[1] + c22 * g[2]) * idet};
        double W[9], W2[9], E[9], T[9], ea, eb, ec;
        hat3(w, W);
        mul33(W, W, W2);
        exp_coeffs(w[0] * w[0] + w[1] * w[1] + w[2] * w[2], &ea, &eb, &ec);
        for (int i = 0; i < 9; ++i) E[i] = ((i % 4 == 0) ? 1.0 : 0.0) + ea * W[i] + eb * W2[i];
        mul33(E, R, T);
        for (int i = 0; i < 9; ++i) R[i] = T[i];
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
// a 6 x mk matrix D, by Householder QR. Returns false under the rank rule
// (min |R_jj| < 1e-14 max |R_jj|) or a non-finite theta.
FRICP_HD inline bool anderson_lstsq(double D[6][kMaxM], double f[6], int mk, double theta[kMaxM]) {
    double Rd[kMaxM];
    for (int j = 0; j < mk; ++j) {
        double col[6];
        for (int i = 0; i < 6; ++i) col[i] = (i < j) ? 0.0 : D[i][j];
        const double nrm2 = dot6(col, col);
        const double nrm = nrm2 > 0.0 ? nrm2 * rsqrt64(nrm2) : 0.0;
        const double alpha = -copysign(nrm, D[j][j]);
        Rd[j] = alpha;
        if (nrm == 0.0) continue;
        double v[6];
        for (int i = 0; i < 6; ++i) v[i] = (i < j) ? 0.0 : D[i][j];
        v[j] -= alpha;
        const double vv = dot6(v, v);
        if (vv == 0.0) continue;
        const double ivv2 = 2.0 * rcp64(vv);
        for (int c = j; c < mk; ++c) {
            double dc[6];
            for (int i = 0; i < 6; ++i) dc[i] = D[i][c];
            const double sc = dot6(v, dc) * ivv2;
            for (int i = j; i < 6; ++i) D[i][c] -= sc * v[i];
        }
        const double sc = dot6(v, f) * ivv2;
        for (int i = j; i < 6; ++i) f[i] -= sc * v[i];
        D[j][j] = alpha;
    }
    double rmax = 0.0, rmin = INFINITY;
    for (int j = 0; j < mk; ++j) {
        rmax = fmax(rmax, fabs(Rd[j]));
        rmin = fmin(rmin, fabs(Rd[j]));
    }
    if (!isfinite(rmax) || rmax == 0.0 || rmin < 1e-14 * rmax) return false;
    for (int j = mk - 1; j >= 0; --j) {
        double acc = f[j];
        for (int c = j + 1; c < mk; ++c) acc -= D[j][c] * theta[c];
        theta[j] = acc * rcp64(D[j][j]);
        if (!isfinite(theta[j])) return false;
    }
    return true;
}

// Cholesky solve of a 6x6 symmetric positive-definite system; false if a pivot
// is not positive and finite. A direction whose row, column and right-hand
// side are all exactly zero is left out and gets x_j = 0: the system of points
// in a plane (z = 0, in-plane normals), where tilting the plane and moving along
// z change no distance, is the 2-D system (Sec. 3 states the problem in R^d).
// 3-D data never has such a direction, and then nothing changes.
FRICP_HD inline bool chol6_solve(const double A_[36], const double b[6], double x[6]) {
    int act[6], na = 0;
    for (int j = 0; j < 6; ++j) {
        bool zero = b[j] == 0.0 && A_[7 * j] == 0.0;   // a zero row has a zero diagonal: test that first
        for (int k = 0; k < 6 && zero; ++k) zero = A_[6 * j + k] == 0.0 && A_[6 * k + j] == 0.0;
        x[j] = 0.0;
        if (!zero) act[na++] = j;
    }
    if (na == 0) return false;
    double L[36];
    for (int i = 0; i < 36; ++i) L[i] = 0.0;
    for (int j = 0; j < na; ++j) {
        double d = A_[7 * act[j]];
        for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
        if (!(d > 0.0) || !isfinite(d)) return false;
        const double il = rsqrt64(d);   // 1 / L_jj
        L[6 * j + j] = il;              // the diagonal holds the reciprocals
        for (int i = j + 1; i < na; ++i) {
            double s = A_[6 * act[i] + act[j]];
            for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
            L[6 * i + j] = s * il;
        }
    }
    double y[6], z[6];
    for (int i = 0; i < na; ++i) {
        double s = b[act[i]];
        for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
        y[i] = s * L[6 * i + i];
    }
    for (int i = na - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < na; ++k) s -= L[6 * k + i] * z[k];
        z[i] = s * L[6 * i + i];
    }
    for (int i = 0; i < na; ++i) x[act[i]] = z[i];
    return true;
}

// Chain matrix K of App. D: the gradient of B_i(xi) = (R p_i + t - q_i) . n_i at
// xi = [delta; u] factors as J_i = K z_i with z_i = [y_i x n_i; n_i], y_i = R p_i,
// because dR/d delta_j = w_j^ R with w_j = (delta_j delta + delta x (I - R) e_j) / |delta|^2
// (so n . (dR/d delta_j) p = w_j . (y x n)). Rows 0..2: [w_j^T, (dt/d delta_j)^T];
// rows 3..5: [0, (dt/du_j)^T], with dt/d delta and dt/du as printed in App. D.
// delta = 0 takes App. D's special case; 0 < |delta| < 1e-6 a second-order series.
FRICP_HD inline void p2pl_chain(const double xi[6], double K[36]) {
    const double *d = xi, *u = xi + 3;
    const double th2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    for (int i = 0; i < 36; ++i) K[i] = 0.0;
    if (th2 == 0.0) {
        for (int j = 0; j < 3; ++j) {
            K[6 * j + j] = 1.0;
            K[6 * (3 + j) + 3 + j] = 1.0;
        }
        return;
    }
    if (th2 < 1e-12) {
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
                K[6 * j + a] = Jl[3 * a + j];                                      // w_j = J_l e_j
                K[6 * j + 3 + a] = 0.5 * exu[a] + (ex_du[a] + d_exu[a]) / 6.0;     // dt/d delta_j
                K[6 * (3 + j) + 3 + a] = Jl[3 * a + j];                            // dt/du_j
            }
        }
        return;
    }
    double T[12];
    const double xr[6] = {d[0], d[1], d[2], 0.0, 0.0, 0.0};
    se3_exp(xr, T);
    const double *R = T;
    double ImR[9], RmI[9];
    for (int i = 0; i < 9; ++i) {
        const double I = (i % 4 == 0) ? 1.0 : 0.0;
        ImR[i] = I - R[i];
        RmI[i] = R[i] - I;
    }
    const double ith2 = rcp64(th2);
    double w[3][3];
    for (int j = 0; j < 3; ++j) {
        const double col[3] = {ImR[j], ImR[3 + j], ImR[6 + j]};
        double cr[3];
        cross3(d, col, cr);
        for (int a = 0; a < 3; ++a) w[j][a] = (d[j] * d[a] + cr[a]) * ith2;
    }
    double Uh[9], M[9];
    hat3(u, Uh);
    mul33(RmI, Uh, M);
    const double du_dot = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
    M[0] += du_dot; M[4] += du_dot; M[8] += du_dot;
    // D_j = (dR/d delta_j) u^ delta = w_j x (R (u x delta))
    double uxd[3], Ruxd[3];
    cross3(u, d, uxd);
    mulv3(R, uxd, Ruxd);
    double Md[3];
    mulv3(M, d, Md);
    double Dt[9];   // Dt[a][j] = dt_a / d delta_j
    for (int j = 0; j < 3; ++j) {
        double Dj[3];
        cross3(w[j], Ruxd, Dj);
        for (int a = 0; a < 3; ++a)
            Dt[3 * a + j] = (M[3 * a + j] + d[a] * u[j] + Dj[a]) * ith2 - 2.0 * ith2 * ith2 * Md[a] * d[j];
    }
    double Dh[9], C[9];
    hat3(d, Dh);
    mul33(ImR, Dh, C);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) C[3 * r + c] = (C[3 * r + c] + d[r] * d[c]) * ith2;
    for (int j = 0; j < 3; ++j)
        for (int a = 0; a < 3; ++a) {
            K[6 * j + a] = w[j][a];
            K[6 * j + 3 + a] = Dt[3 * a + j];
            K[6 * (3 + j) + 3 + a] = C[3 * a + j];
        }
}

}  // namespace fricp
