// Host build of the device small-algebra routines (they are __host__ __device__),
// exported with C linkage so the CPU tests can compare them with numpy/scipy.
#include "../paper_2007_07627_gb300/csrc/linalg.cuh"

extern "C" {

int h_procrustes_rotation(const double *H, double *R) { return fricp::procrustes_rotation(H, R) ? 1 : 0; }

void h_se3_exp(const double *xi, double *T) { fricp::se3_exp(xi, T); }

void h_se3_log(const double *T, double *xi) { fricp::se3_log(T, xi); }

int h_anderson_lstsq(const double *D_in, const double *f_in, int mk, double *theta) {
    double D[6][fricp::kMaxM], f[6];
    for (int i = 0; i < 6; ++i) {
        f[i] = f_in[i];
        for (int j = 0; j < mk; ++j) D[i][j] = D_in[i * mk + j];
    }
    return fricp::anderson_lstsq(D, f, mk, theta) ? 1 : 0;
}

int h_chol6_solve(const double *A, const double *b, double *x) { return fricp::chol6_solve(A, b, x) ? 1 : 0; }

void h_p2pl_chain(const double *xi, double *K) { fricp::p2pl_chain(xi, K); }
}
