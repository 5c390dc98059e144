/*
 * FP64 brute-force point queries for the oracle of "Fast and Robust Iterative
 * Closest Point" (Zhang, Yao, Deng, 2020).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load this library. It shares no code with the CUDA path.
 *
 * oracle_closest   : the correspondence step, Sec. 3 Eq. (3) (closest point of
 *                    each transformed source point in Q), by exhaustive search.
 *                    Ties go to the lowest target index (first one met).
 *                    Also returns the second-smallest squared distance, used by
 *                    the parity tests' near-tie rule.
 * oracle_knn_self  : the k nearest points of every q_i within Q, q_i itself
 *                    excluded (the six-nearest-point statistic of Sec. 4.3 and
 *                    Sec. 5), by exhaustive search, ascending (d^2, index).
 * oracle_knn_all   : the same with q_i itself included (the neighbourhoods of
 *                    the normal estimate of Sec. 6).
 * oracle_knn_query : the k nearest points of Q of arbitrary query points x
 *                    (a point of Q queried at its own position finds itself).
 *
 * Compiled with -ffp-contract=off so x86-64 and AArch64 give identical bits.
 */
#include <math.h>
#include <stdint.h>

void oracle_closest(const double *x, int64_t m, const double *q, int64_t n,
                    int64_t *idx, double *d2, double *d2_second)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < m; ++i) {
        const double x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
        double best = INFINITY, second = INFINITY;
        int64_t arg = -1;
        for (int64_t j = 0; j < n; ++j) {
            const double a = x0 - q[3 * j];
            const double b = x1 - q[3 * j + 1];
            const double c = x2 - q[3 * j + 2];
            const double d = a * a + b * b + c * c;
            if (d < best) {
                second = best;
                best = d;
                arg = j;
            } else if (d < second) {
                second = d;
            }
        }
        idx[i] = arg;
        d2[i] = best;
        d2_second[i] = second;
    }
}

void oracle_knn_self(const double *q, int64_t n, int k, int64_t *idx, double *d2)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < n; ++i) {
        double *bd = d2 + i * k;
        int64_t *bi = idx + i * k;
        for (int s = 0; s < k; ++s) {
            bd[s] = INFINITY;
            bi[s] = -1;
        }
        const double x0 = q[3 * i], x1 = q[3 * i + 1], x2 = q[3 * i + 2];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            const double a = q[3 * j] - x0;
            const double b = q[3 * j + 1] - x1;
            const double c = q[3 * j + 2] - x2;
            const double d = a * a + b * b + c * c;
            if (!(d < bd[k - 1]))
                continue;
            /* insert after every entry with an equal or smaller distance */
            int s = k - 1;
            while (s > 0 && bd[s - 1] > d) {
                bd[s] = bd[s - 1];
                bi[s] = bi[s - 1];
                --s;
            }
            bd[s] = d;
            bi[s] = j;
        }
    }
}

void oracle_knn_all(const double *q, int64_t n, int k, int64_t *idx, double *d2)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < n; ++i) {
        double *bd = d2 + i * k;
        int64_t *bi = idx + i * k;
        for (int s = 0; s < k; ++s) {
            bd[s] = INFINITY;
            bi[s] = -1;
        }
        const double x0 = q[3 * i], x1 = q[3 * i + 1], x2 = q[3 * i + 2];
        for (int64_t j = 0; j < n; ++j) {
            const double a = q[3 * j] - x0;
            const double b = q[3 * j + 1] - x1;
            const double c = q[3 * j + 2] - x2;
            const double d = a * a + b * b + c * c;
            if (!(d < bd[k - 1]))
                continue;
            int s = k - 1;
            while (s > 0 && bd[s - 1] > d) {
                bd[s] = bd[s - 1];
                bi[s] = bi[s - 1];
                --s;
            }
            bd[s] = d;
            bi[s] = j;
        }
    }
}

void oracle_knn_query(const double *x, int64_t m, const double *q, int64_t n, int k, int64_t *idx, double *d2)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < m; ++i) {
        double *bd = d2 + i * k;
        int64_t *bi = idx + i * k;
        for (int s = 0; s < k; ++s) {
            bd[s] = INFINITY;
            bi[s] = -1;
        }
        const double x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
        for (int64_t j = 0; j < n; ++j) {
            const double a = q[3 * j] - x0;
            const double b = q[3 * j + 1] - x1;
            const double c = q[3 * j + 2] - x2;
            const double d = a * a + b * b + c * c;
            if (!(d < bd[k - 1]))
                continue;
            int s = k - 1;
            while (s > 0 && bd[s - 1] > d) {
                bd[s] = bd[s - 1];
                bi[s] = bi[s - 1];
                --s;
            }
            bd[s] = d;
            bi[s] = j;
        }
    }
}
