// Oriented bounding box of a bucket of target points, and the float distance
// test the closest-point search runs against it. Host and device code: the
// kernels build and test the boxes with these functions, and a CPU test runs
// the same functions against exact FP64 distances.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#ifndef FRICP_HD
#define FRICP_HD __host__ __device__
#endif

namespace fricp {

// v rounded up to float.
FRICP_HD inline float f32_round_up(double v) {
#ifdef __CUDA_ARCH__
    return __double2float_ru(v);
#else
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
#endif
}

FRICP_HD inline float f32_rsqrt(float x) {
#ifdef __CUDA_ARCH__
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}

// Eigenvectors of the symmetric 3x3 matrix A (cyclic Jacobi rotations, float):
// the columns of V. Only the tightness of the oriented boxes depends on them.
FRICP_HD inline void jacobi3f(float A[3][3], float V[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0f : 0.0f;
    for (int sweep = 0; sweep < 8; ++sweep) {
        const float off = fabsf(A[0][1]) + fabsf(A[0][2]) + fabsf(A[1][2]);
        const float dia = fabsf(A[0][0]) + fabsf(A[1][1]) + fabsf(A[2][2]);
        if (!(off > 1e-7f * dia)) break;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0f) continue;
                const float theta = (A[q][q] - A[p][p]) / (2.0f * A[p][q]);
                const float t = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
                const float c = f32_rsqrt(fmaf(t, t, 1.0f)), sn = t * c;
                for (int k = 0; k < 3; ++k) {   // A <- A J (columns p, q)
                    const float akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {   // A <- J^T A (rows p, q)
                    const float apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {   // V <- V J
                    const float vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
        }
    }
}

// Oriented box of the cnt >= 1 points p[0 .. cnt) (.w unused), written as
// out[0 .. 3] = (c, h0) (a0, h1) (a1, h2) (a2, r): axes along the points'
// principal directions, made orthonormal in FP64 and rounded to float (those
// float axes are what the box is exact for; a set that is not orthonormal to
// 1e-6 falls back to the coordinate axes); the points' extents along them in
// FP64 about a float centre c; the half-extents h widened by 1e-6 relative, 2e-6
// of the radius r and 1e-12 of the coordinates' magnitude, then rounded up to
// float.
FRICP_HD inline void obb_fit(const float4 *p, int cnt, float4 out[4]) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < cnt; ++j) {
        s[0] += p[j].x;
        s[1] += p[j].y;
        s[2] += p[j].z;
    }
    const float c0[3] = {(float)(s[0] / cnt), (float)(s[1] / cnt), (float)(s[2] / cnt)};
    float A[3][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    for (int j = 0; j < cnt; ++j) {
        const float d[3] = {p[j].x - c0[0], p[j].y - c0[1], p[j].z - c0[2]};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[a][b] = fmaf(d[a], d[b], A[a][b]);
    }
    float V[3][3];
    jacobi3f(A, V);
    // Gram-Schmidt in FP64 on the first two eigenvectors, third = cross product
    double ax[3][3];
    {
        double v0[3] = {V[0][0], V[1][0], V[2][0]}, v1[3] = {V[0][1], V[1][1], V[2][1]};
        const double n0 = sqrt(v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2]);
        for (int a = 0; a < 3; ++a) v0[a] /= n0;
        const double d01 = v0[0] * v1[0] + v0[1] * v1[1] + v0[2] * v1[2];
        for (int a = 0; a < 3; ++a) v1[a] -= d01 * v0[a];
        const double n1 = sqrt(v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]);
        for (int a = 0; a < 3; ++a) v1[a] /= n1;
        const double v2[3] = {v0[1] * v1[2] - v0[2] * v1[1], v0[2] * v1[0] - v0[0] * v1[2],
                              v0[0] * v1[1] - v0[1] * v1[0]};
        for (int a = 0; a < 3; ++a) {
            ax[0][a] = (double)(float)v0[a];
            ax[1][a] = (double)(float)v1[a];
            ax[2][a] = (double)(float)v2[a];
        }
    }
    bool ortho = true;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double g = ax[a][0] * ax[b][0] + ax[a][1] * ax[b][1] + ax[a][2] * ax[b][2];
            if (!(fabs(g - (a == b ? 1.0 : 0.0)) <= 1e-6)) ortho = false;
        }
    if (!ortho)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) ax[a][b] = a == b ? 1.0 : 0.0;
    // extents about c0, then about the float centre of the box
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = 0; j < cnt; ++j) {
        const double d[3] = {(double)p[j].x - c0[0], (double)p[j].y - c0[1], (double)p[j].z - c0[2]};
        for (int k = 0; k < 3; ++k) {
            const double u = ax[k][0] * d[0] + ax[k][1] * d[1] + ax[k][2] * d[2];
            lo[k] = fmin(lo[k], u);
            hi[k] = fmax(hi[k], u);
        }
    }
    float c[3];
    for (int a = 0; a < 3; ++a) {
        double v = c0[a];
        for (int k = 0; k < 3; ++k) v += 0.5 * (lo[k] + hi[k]) * ax[k][a];
        c[a] = (float)v;
    }
    double h[3] = {0.0, 0.0, 0.0}, r2 = 0.0;
    for (int j = 0; j < cnt; ++j) {
        const double d[3] = {(double)p[j].x - c[0], (double)p[j].y - c[1], (double)p[j].z - c[2]};
        for (int k = 0; k < 3; ++k) h[k] = fmax(h[k], fabs(ax[k][0] * d[0] + ax[k][1] * d[1] + ax[k][2] * d[2]));
        r2 = fmax(r2, d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    const double r = sqrt(r2);
    const double mag = fmax(fmax(fabs((double)c[0]), fabs((double)c[1])), fabs((double)c[2])) + r;
    float hf[3];
    for (int k = 0; k < 3; ++k) hf[k] = f32_round_up(h[k] * (1.0 + 1e-6) + 2e-6 * r + 1e-12 * mag);
    out[0] = make_float4(c[0], c[1], c[2], hf[0]);
    out[1] = make_float4((float)ax[0][0], (float)ax[0][1], (float)ax[0][2], hf[1]);
    out[2] = make_float4((float)ax[1][0], (float)ax[1][1], (float)ax[1][2], hf[2]);
    out[3] = make_float4((float)ax[2][0], (float)ax[2][1], (float)ax[2][2], (float)r);
}

// Squared distance from x = xh + xl to the box (c, h0) (a0, h1) (a1, h2) (a2, .),
// in float. Against the widening of obb_fit, the float rounding of
// u = A ((xh - c) + xl) (at most ~5.2e-7 of |x - c| per axis) leaves the result
// at most (1 + 8e-6) times the squared distance to the nearest of the box's
// points.
FRICP_HD inline float obb_eval(float4 c, float4 a0, float4 a1, float4 a2, const float xh[3], const float xl[3]) {
    const float dx = (xh[0] - c.x) + xl[0];
    const float dy = (xh[1] - c.y) + xl[1];
    const float dz = (xh[2] - c.z) + xl[2];
    const float e0 = fmaxf(fabsf(fmaf(a0.z, dz, fmaf(a0.y, dy, a0.x * dx))) - c.w, 0.0f);
    const float e1 = fmaxf(fabsf(fmaf(a1.z, dz, fmaf(a1.y, dy, a1.x * dx))) - a0.w, 0.0f);
    const float e2 = fmaxf(fabsf(fmaf(a2.z, dz, fmaf(a2.y, dy, a2.x * dx))) - a1.w, 0.0f);
    return fmaf(e2, e2, fmaf(e1, e1, e0 * e0));
}

}  // namespace fricp
