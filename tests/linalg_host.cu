// Host build of the solver's small-algebra routines (they are __host__ __device__
// and run on a Team; on the host a team is one lane), exported with C linkage so
// the CPU tests can compare them with numpy/scipy.
#include "../paper_2007_07627_gb300/csrc/linalg.cuh"

namespace {
struct HostTeam {
    double sh[fricp::kTeamScratch];
    fricp::Team tm{sh};
};
}  // namespace

extern "C" {

int h_procrustes_rotation(const double *H, double *R) {
    HostTeam t;
    for (int i = 0; i < 9; ++i) t.sh[i] = H[i];
    const bool ok = fricp::procrustes_rotation(t.tm, t.sh, t.sh + 16, t.sh + 32);
    for (int i = 0; i < 9; ++i) R[i] = t.sh[16 + i];
    return ok ? 1 : 0;
}

void h_se3_exp(const double *xi, double *T) {
    HostTeam t;
    const double x[6] = {xi[0], xi[1], xi[2], xi[3], xi[4], xi[5]};
    fricp::se3_exp(t.tm, x, t.sh, t.sh + 16);
    for (int i = 0; i < 12; ++i) T[i] = t.sh[i];
}

void h_se3_log(const double *T, double *xi) {
    HostTeam t;
    for (int i = 0; i < 12; ++i) t.sh[i] = T[i];
    double x[6];
    fricp::se3_log(t.tm, t.sh, x, t.sh + 16);
    for (int i = 0; i < 6; ++i) xi[i] = x[i];
}

int h_anderson_lstsq(const double *D_in, const double *f_in, int mk, double *theta) {
    HostTeam t;
    double *Dm = t.sh;
    for (int i = 0; i < 6; ++i) {
        Dm[6 * fricp::kMaxM + i] = f_in[i];
        for (int j = 0; j < mk; ++j) Dm[6 * j + i] = D_in[i * mk + j];
    }
    double th[fricp::kMaxM];
    const bool ok = fricp::anderson_lstsq(t.tm, Dm, mk, th, t.sh + 48);
    for (int j = 0; j < mk; ++j) theta[j] = th[j];
    return ok ? 1 : 0;
}

int h_chol6_solve(const double *A, const double *b, double *x) {
    HostTeam t;
    for (int i = 0; i < 36; ++i) t.sh[i] = A[i];
    for (int i = 0; i < 6; ++i) t.sh[36 + i] = b[i];
    double y[6];
    const bool ok = fricp::chol6_solve(t.tm, t.sh, t.sh + 36, y, t.sh + 48);
    for (int i = 0; i < 6; ++i) x[i] = y[i];
    return ok ? 1 : 0;
}

void h_p2pl_chain(const double *xi, double *K) {
    HostTeam t;
    const double x[6] = {xi[0], xi[1], xi[2], xi[3], xi[4], xi[5]};
    fricp::p2pl_chain(t.tm, x, t.sh, t.sh + 40);
    for (int i = 0; i < 36; ++i) K[i] = t.sh[i];
}
}
