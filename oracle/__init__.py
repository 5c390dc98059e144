"""FP64 CPU oracle for "Fast and Robust Iterative Closest Point"
(J. Zhang, Y. Yao, B. Deng; IEEE TPAMI 2021, arXiv 2007.07627).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline and --impl reference legs may import this package. It shares no
code with the CUDA path (paper_2007_07627_gb300) and imports nothing from it.

It is a plain, slow restatement of the paper in FP64 on the float32 inputs
widened to float64:
  * correspondence step (Sec. 3, Eq. 3) by exhaustive search (nn_bruteforce.c),
    or, for full-size inputs, a library k-d tree query whose result is pinned
    to be the same (closest_kdtree);
  * closed-form weighted rigid alignment (Sec. 3 Eq. 4 and Sec. 4.3 Eq. 12) via
    numpy's SVD;
  * exp / log on SE(3) (Sec. 4.2, Eqs. 8-9; App. A) as scipy's matrix
    exponential / principal matrix logarithm, which is what App. A computes for
    rotation angles below pi;
  * Anderson acceleration (Sec. 4.1, Eq. 6) with numpy's Householder QR;
  * Algorithm 1 (Welsch point-to-point, and with psi -> squared distance,
    w == 1 and a single stage, the accelerated point-to-point "Fast ICP");
  * Algorithm 2 (Welsch point-to-plane) with the App. D gradient, and the
    plain point-to-plane objective of Eq. (15) under it;
  * the Welsch-robust symmetric objective Sec. 7 proposes as future work, read
    as Algorithm 2 on the residual of symmetric_residual;
  * the nu_max / nu_min rules (Sec. 4.3, Sec. 5, App. C);
  * normals from the k nearest neighbours (Sec. 6, estimate_normals).
Where the paper is silent, garbled or inconsistent the reading taken is a named
constant or a commented branch below, each citing the passage it reads.

Pins (tests/test_oracle_pins.py, and tests/test_golden_parameters.py for the
values the paper prints) tie every function here to something other than
itself. The energy/iteration trajectory of a whole registration at workload
scale is "parity unpinned" beyond these per-step pins: the paper prints no
worked example and its datasets are not available.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import pathlib
import subprocess
import tempfile

import numpy as np
import scipy.linalg as sla

_HERE = pathlib.Path(__file__).resolve().parent
_SO = _HERE / "_nn_bruteforce.so"
_lib = None

# ---------------------------------------------------------------------------
# Readings of the paper (each one listed with its justification in the design
# notes). Names follow the paper.
# ---------------------------------------------------------------------------
#: Sec. 4.1: "F^(k) = G(x^(k))" is read as F^(k) = G(x^(k)) - x^(k), the
#: residual F(x) = G(x) - x defined in the same sentence (and Alg. 1/2's use).
#: Alg. 1/2 sum the AA correction to m; read m_k (the LS has m_k unknowns).
#: AA least squares is skipped (plain G^(k) taken) when the QR of the
#: difference matrix is rank deficient: min|R_jj| < AA_RANK_TOL * max|R_jj|.
AA_RANK_TOL = 1e-14
#: Alg. 2 line search never updates tau or l: read tau <- tau/2, l <- l+1.
#: l_max is not given: default MAX_LINE_SEARCH.
MAX_LINE_SEARCH = 10
#: Below this |delta| the App. D closed forms divide tiny by tiny; a series is
#: used instead (exactly delta = 0 keeps App. D's own special case).
SMALL_DELTA = 1e-6
#: nu_min is clamped from below (a perfectly flat target gives H_Q = 0).
NU_MIN_FLOOR = 1e-6


class Degenerate(RuntimeError):
    """All Welsch weights vanished, or the point-to-plane normal matrix is singular."""


# ---------------------------------------------------------------------------
# Brute-force queries (C, OpenMP)
# ---------------------------------------------------------------------------

def build(force: bool = False) -> pathlib.Path:
    """Compile nn_bruteforce.c with gcc (plain C, OpenMP, no FP contraction)."""
    if _SO.exists() and not force and _SO.stat().st_mtime >= (_HERE / "nn_bruteforce.c").stat().st_mtime:
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=str(_HERE))
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           str(_HERE / "nn_bruteforce.c"), "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_closest.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64, ip, dp, dp]
        lib.oracle_closest.restype = None
        lib.oracle_knn_self.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip, dp]
        lib.oracle_knn_self.restype = None
        lib.oracle_knn_all.argtypes = [dp, ctypes.c_int64, ctypes.c_int, ip, dp]
        lib.oracle_knn_all.restype = None
        lib.oracle_knn_query.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64, ctypes.c_int, ip, dp]
        lib.oracle_knn_query.restype = None
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def closest(X: np.ndarray, Q: np.ndarray):
    """Sec. 3 Eq. (3): index of the closest q in Q for every row of X.

    Returns (idx int64[m], d2 float64[m], d2_second float64[m]); ties go to the
    lowest index of Q.
    """
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    m, n = X.shape[0], Q.shape[0]
    idx = np.empty(m, np.int64)
    d2 = np.empty(m, np.float64)
    d2s = np.empty(m, np.float64)
    if m:
        lib.oracle_closest(_dp(X), m, _dp(Q), n, _ip(idx), _dp(d2), _dp(d2s))
    return idx, d2, d2s


def closest_kdtree(X: np.ndarray, Q: np.ndarray, tree=None, k: int = 8):
    """Sec. 3 Eq. (3) through a library nearest-neighbour query, for inputs too
    large for the exhaustive search: scipy's k-d tree proposes the k nearest
    points of Q for every row of X, each squared distance is then recomputed
    exactly as `closest` computes it ((a*a + b*b) + c*c in FP64), and the
    minimum is taken with ties to the lowest index. The result equals
    `closest`, bit for bit, whenever fewer than k points of Q lie within
    rounding of a row's minimum (pinned against it on random, duplicated and
    tied inputs). Returns (idx, d2, d2_second) like `closest`; `tree`: a
    scipy.spatial.cKDTree of Q, built here when not given."""
    from scipy.spatial import cKDTree
    X = np.ascontiguousarray(X, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    m, n = X.shape[0], Q.shape[0]
    if m == 0:
        return np.empty(0, np.int64), np.empty(0), np.empty(0)
    if tree is None:
        tree = cKDTree(Q)
    kk = min(k, n)
    _, cand = tree.query(X, k=kk, workers=-1)
    cand = np.asarray(cand, dtype=np.int64).reshape(m, kk)
    diff = X[:, None, :] - Q[cand]
    d2 = (diff[..., 0] * diff[..., 0] + diff[..., 1] * diff[..., 1]) + diff[..., 2] * diff[..., 2]
    # lexicographic (d2, index) order of each row's candidates
    o = np.argsort(cand, axis=1, kind="stable")
    cand = np.take_along_axis(cand, o, 1)
    d2 = np.take_along_axis(d2, o, 1)
    o = np.argsort(d2, axis=1, kind="stable")
    cand = np.take_along_axis(cand, o, 1)
    d2 = np.take_along_axis(d2, o, 1)
    second = d2[:, 1] if kk > 1 else np.full(m, np.inf)
    return cand[:, 0].copy(), d2[:, 0].copy(), second.copy()


def nn_function(Q: np.ndarray, method: str = "bruteforce"):
    """The correspondence step against a fixed Q (Sec. 3: Q does not change over
    a registration): `closest` (exhaustive, the definition) or `closest_kdtree`
    (a library query, equal to it; its tree built once here)."""
    if method == "bruteforce":
        return lambda X: closest(X, Q)
    if method == "kdtree":
        from scipy.spatial import cKDTree
        Qc = np.ascontiguousarray(Q, dtype=np.float64)
        tree = cKDTree(Qc)
        return lambda X: closest_kdtree(X, Qc, tree)
    raise ValueError(method)


def knn_self(Q: np.ndarray, k: int):
    """k nearest points of each q_i in Q with q_i itself excluded (Sec. 4.3)."""
    lib = _load()
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = Q.shape[0]
    idx = np.empty((n, k), np.int64)
    d2 = np.empty((n, k), np.float64)
    if n:
        lib.oracle_knn_self(_dp(Q), n, k, _ip(idx), _dp(d2))
    return idx, d2


def knn_all(Q: np.ndarray, k: int):
    """k nearest points of each q_i in Q, q_i itself included (Sec. 6 normals)."""
    lib = _load()
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = Q.shape[0]
    k = min(k, n)
    idx = np.empty((n, k), np.int64)
    d2 = np.empty((n, k), np.float64)
    if n:
        lib.oracle_knn_all(_dp(Q), n, k, _ip(idx), _dp(d2))
    return idx, d2


def knn_query(X: np.ndarray, Q: np.ndarray, k: int):
    """k nearest points of Q for each row of X, ascending (d^2, index of Q)."""
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    m, n = X.shape[0], Q.shape[0]
    k = min(k, n)
    idx = np.empty((m, k), np.int64)
    d2 = np.empty((m, k), np.float64)
    if m:
        lib.oracle_knn_query(_dp(X), m, _dp(Q), n, k, _ip(idx), _dp(d2))
    return idx, d2


def estimate_normals(Q: np.ndarray, k: int = 30, viewpoint=None, rows=None) -> np.ndarray:
    """Normals of a point set where the surface is unknown (Sec. 6: the paper uses
    PCL's estimate over 30 nearest neighbours). Reading: the neighbourhood of q_i is
    its k nearest points in Q, q_i included, ties to the lower index; the normal
    is the unit eigenvector of the smallest eigenvalue of the neighbourhood's
    covariance (1/k) sum (q_j - c)(q_j - c)^T about its centroid c, turned so that
    n . (viewpoint - q_i) >= 0 (viewpoint: the origin when not given). rows: only
    those points' normals (all when None)."""
    Q = np.asarray(Q, dtype=np.float64)
    v = np.zeros(3) if viewpoint is None else np.asarray(viewpoint, dtype=np.float64)
    if rows is None:
        idx, _ = knn_all(Q, k)
        at = Q
    else:
        at = Q[np.asarray(rows)]
        idx, _ = knn_query(at, Q, k)
    nb = Q[idx]                                       # [m, k, 3]
    c = nb.mean(axis=1, keepdims=True)
    C = np.einsum("nki,nkj->nij", nb - c, nb - c) / nb.shape[1]
    _, vecs = np.linalg.eigh(C)                       # ascending eigenvalues
    nrm = vecs[:, :, 0]
    flip = np.einsum("nd,nd->n", nrm, v[None, :] - at) < 0.0
    nrm[flip] *= -1.0
    return nrm


# ---------------------------------------------------------------------------
# Normalization (Sec. 6 set-up)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Normalization:
    """One similarity x -> s (x - c) applied to both P and Q.

    Reading of Sec. 6 ("aligning the centroids ... scaling such that the bounding
    box has diagonal length 1"): c is the centroid of Q, s the inverse diagonal of
    the bounding box of P u Q. The same map on both sets keeps the initial
    transformation's meaning, so an identity start stays the identity.
    """
    c: np.ndarray
    s: float

    def fwd(self, X):
        return self.s * (X - self.c)

    def T_to_normalized(self, T):
        Tn = np.eye(4)
        R, t = T[:3, :3], T[:3, 3]
        Tn[:3, :3] = R
        Tn[:3, 3] = self.s * (R @ self.c + t - self.c)
        return Tn

    def T_to_original(self, Tn):
        T = np.eye(4)
        R, t = Tn[:3, :3], Tn[:3, 3]
        T[:3, :3] = R
        T[:3, 3] = t / self.s + self.c - R @ self.c
        return T


def normalization(P: np.ndarray, Q: np.ndarray) -> Normalization:
    c = Q.mean(axis=0)
    lo = np.minimum(P.min(axis=0), Q.min(axis=0))
    hi = np.maximum(P.max(axis=0), Q.max(axis=0))
    return Normalization(c=c, s=1.0 / float(np.linalg.norm(hi - lo)))


# ---------------------------------------------------------------------------
# Welsch's function and its surrogate (Sec. 4.3, Eqs. 10-11; App. B)
# ---------------------------------------------------------------------------

def welsch(x, nu):
    """psi_nu(x) = 1 - exp(-x^2 / (2 nu^2))  (Eq. 10)."""
    x = np.asarray(x, dtype=np.float64)
    return 1.0 - np.exp(-(x * x) / (2.0 * nu * nu))


def welsch_surrogate(x, y, nu):
    """chi_nu(x | y) = psi_nu(y) + (x^2 - y^2)/(2 nu^2) exp(-y^2/(2 nu^2))  (Eq. 11)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return welsch(y, nu) + (x * x - y * y) / (2.0 * nu * nu) * np.exp(-(y * y) / (2.0 * nu * nu))


# ---------------------------------------------------------------------------
# SE(3) (Sec. 4.2 Eqs. 7-9, App. A)
# ---------------------------------------------------------------------------

def hat(a) -> np.ndarray:
    """a^ : the skew matrix with a^ b = a x b (App. D)."""
    a1, a2, a3 = float(a[0]), float(a[1]), float(a[2])
    return np.array([[0.0, -a3, a2], [a3, 0.0, -a1], [-a2, a1, 0.0]])


def se3_matrix(xi) -> np.ndarray:
    """The se(3) matrix [[S, u], [0, 0]] of Eq. (8) for xi = [delta; u], S = delta^."""
    X = np.zeros((4, 4))
    X[:3, :3] = hat(xi[:3])
    X[:3, 3] = xi[3:6]
    return X


def se3_vee(X) -> np.ndarray:
    return np.array([X[2, 1], X[0, 2], X[1, 0], X[0, 3], X[1, 3], X[2, 3]])


def se3_exp(X: np.ndarray) -> np.ndarray:
    """Eq. (9): T = exp(X), the matrix exponential of an se(3) matrix."""
    return sla.expm(X)


def se3_log(T: np.ndarray) -> np.ndarray:
    """App. A: log(T), the principal matrix logarithm of T in SE(3).

    For rotation angles in [0, pi) the real-Schur construction of App. A returns
    the principal logarithm, which is what scipy's logm computes.
    """
    L = sla.logm(T)
    if np.iscomplexobj(L):
        if np.abs(L.imag).max() > 1e-12:
            raise ValueError("rotation angle at pi: logarithm not unique")
        L = L.real
    L[3, :] = 0.0
    return L


def apply(T, X):
    return X @ T[:3, :3].T + T[:3, 3]


# ---------------------------------------------------------------------------
# Alignment step: weighted Procrustes (Eq. 4, Eq. 12)
# ---------------------------------------------------------------------------

def weighted_procrustes(P: np.ndarray, Qh: np.ndarray, w: np.ndarray) -> np.ndarray:
    """argmin over SO(3) x R^3 of sum_i w_i ||R p_i + t - q_i||^2, closed form via SVD."""
    W = float(w.sum())
    if not (W > 0.0) or not math.isfinite(W):
        raise Degenerate("sum of weights is zero")
    pbar = (w[:, None] * P).sum(axis=0) / W
    qbar = (w[:, None] * Qh).sum(axis=0) / W
    H = ((P - pbar) * w[:, None]).T @ (Qh - qbar)   # sum_i w_i (p_i - pbar)(q_i - qbar)^T
    U, _, Vt = np.linalg.svd(H)
    V = Vt.T
    d = 1.0 if np.linalg.det(V @ U.T) >= 0.0 else -1.0   # reflection fix
    R = V @ np.diag([1.0, 1.0, d]) @ U.T
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = qbar - R @ pbar
    return T


# ---------------------------------------------------------------------------
# Anderson acceleration (Sec. 4.1 Eq. 6)
# ---------------------------------------------------------------------------

def anderson_theta(Fk: np.ndarray, dF: np.ndarray):
    """theta* = argmin || F^(k) - sum_j theta_j dF_j ||_2 by Householder QR.

    dF has one column per j = 1..m_k: F^(k-j+1) - F^(k-j). Returns None when
    the rank rule (AA_RANK_TOL) rejects the problem or theta is not finite.
    """
    if dF.shape[1] == 0:
        return None
    Qm, Rm = np.linalg.qr(dF)
    dg = np.abs(np.diag(Rm))
    if not np.all(np.isfinite(dg)) or dg.max() == 0.0 or dg.min() < AA_RANK_TOL * dg.max():
        return None
    theta = sla.solve_triangular(Rm, Qm.T @ Fk)
    if not np.all(np.isfinite(theta)):
        return None
    return theta


# ---------------------------------------------------------------------------
# nu rules (Sec. 4.3, Sec. 5, App. C)
# ---------------------------------------------------------------------------

def _median_of_six(v):
    """Median of six values: mean of the 3rd and 4th smallest (numpy's even-count rule)."""
    return np.median(v, axis=1)


def nu_min_point_to_point(Qn: np.ndarray) -> float:
    """nu_min = E_Q / (3 sqrt 3); E_Q = median over q of the median distance to its 6 NN."""
    _, d2 = knn_self(Qn, 6)
    return float(np.median(_median_of_six(np.sqrt(d2)))) / (3.0 * math.sqrt(3.0))


def nu_min_point_to_plane(Qn: np.ndarray, Nq: np.ndarray) -> float:
    """nu_min = H_Q / 6; H_Q = median over q of the median |(q_j - q) . n_q| over its 6 NN (Sec. 5)."""
    idx, _ = knn_self(Qn, 6)
    h = np.abs(np.einsum("nkd,nd->nk", Qn[idx] - Qn[:, None, :], Nq))
    return float(np.median(_median_of_six(h))) / 6.0


# ---------------------------------------------------------------------------
# Parameters and results
# ---------------------------------------------------------------------------

VARIANTS = ("p2p", "p2p_welsch", "p2pl_welsch", "p2pl", "sym_welsch")


@dataclasses.dataclass
class Params:
    variant: str = "p2p_welsch"
    anderson_m: int = 5            # m = 5 (Sec. 4.2)
    max_iters: int = 1000          # I_nu for point-to-point (Sec. 4.3)
    p2pl_iters_first: int = 6      # I_nu at nu_max for point-to-plane (Sec. 5)
    p2pl_iters_cap: int = 10       # +1 per stage, at most 10 (Sec. 5)
    max_line_search: int = MAX_LINE_SEARCH
    eps: float = 1e-5              # epsilon_nu (Sec. 4.3, Sec. 5)
    nu_max: float = 0.0            # <= 0: paper rule
    nu_min: float = 0.0            # <= 0: paper rule
    nu_min_floor: float = NU_MIN_FLOOR
    # Sensitivity probe, off by default (0.0 leaves every result unchanged):
    # each alignment result (T' of Eq. 4 / Eq. 12, xi* of Eq. 19) is moved by a
    # seeded rigid perturbation of this size in normalised units, the scale of
    # the rounding in which two correct FP64 implementations differ. Runs with
    # it on show how far the iteration amplifies rounding on a given input.
    solve_jitter: float = 0.0
    jitter_seed: int = 0
    # Correspondence step: "bruteforce" (exhaustive, the definition) or
    # "kdtree" (closest_kdtree: a library query with the same result, for
    # full-size inputs).
    nn: str = "bruteforce"


def _jitter(params: Params):
    """(perturb_T, perturb_xi) for Params.solve_jitter; identities when it is 0."""
    if params.solve_jitter == 0.0:
        return (lambda T: T), (lambda xi: xi)
    g = np.random.default_rng(params.jitter_seed)
    eps = params.solve_jitter
    return (lambda T: se3_exp(se3_matrix(eps * g.standard_normal(6))) @ T), \
           (lambda xi: xi + eps * g.standard_normal(6))


def _result(nz, Tn, c, nu_max, nu_min, E, trace, status="ok"):
    T = nz.T_to_original(Tn)
    out = dict(R=T[:3, :3].copy(), t=T[:3, 3].copy(), T_normalized=Tn, s=nz.s, c=nz.c,
               nu_max=nu_max, nu_min=nu_min, final_energy=E, trace=np.array(trace),
               status=status)
    out.update(c)
    return out


def _counters():
    return dict(iterations=0, corr_passes=0, aa_accepted=0, reverts=0,
                line_search_trials=0, stages=0)


# ---------------------------------------------------------------------------
# Algorithm 1: robust point-to-point ICP with AA (and "Fast ICP")
# ---------------------------------------------------------------------------

def register_point_to_point(P32, Q32, params: Params, T0=None) -> dict:
    """Algorithm 1. params.variant 'p2p_welsch' (Welsch, nu stages) or 'p2p'
    (Fast ICP: energy sum D_i^2, weights 1, a single stage)."""
    robust = params.variant == "p2p_welsch"
    P = np.asarray(P32, dtype=np.float64)
    Q = np.asarray(Q32, dtype=np.float64)
    nz = normalization(P, Q)
    Pn, Qn = nz.fwd(P), nz.fwd(Q)
    cnt = _counters()
    trace = []
    m = params.anderson_m

    nn = nn_function(Qn, params.nn)

    def corr(T):
        cnt["corr_passes"] += 1
        idx, d2, _ = nn(apply(T, Pn))
        return idx, d2

    def energy(C, nu):
        d2 = C[1]
        return float(welsch(np.sqrt(d2), nu).sum()) if robust else float(d2.sum())

    jit_T, _ = _jitter(params)

    def align(C, nu):
        idx, d2 = C
        w = np.exp(-d2 / (2.0 * nu * nu)) if robust else np.ones_like(d2)
        return jit_T(weighted_procrustes(Pn, Qn[idx], w))

    T_prev = np.eye(4) if T0 is None else nz.T_to_normalized(np.asarray(T0, np.float64))
    C_prev = corr(T_prev)                                     # Q^(0)
    if robust:
        nu_max = params.nu_max if params.nu_max > 0 else 3.0 * float(np.median(np.sqrt(C_prev[1])))
        nu_min = params.nu_min if params.nu_min > 0 else nu_min_point_to_point(Qn)
        nu_min = max(nu_min, params.nu_min_floor)
        nu_max = max(nu_max, nu_min)          # nu_max <= nu_min: one stage at nu_min
    else:
        nu_max = nu_min = 1.0                 # unused; a single stage
    nu = nu_max
    E_prev = math.inf
    Tk = T_prev
    try:
        while True:
            cnt["stages"] += 1
            E_prev = math.inf
            Tp = align(C_prev, nu)                       # T' from T^(k-1)
            Tk, Ck = Tp, corr(Tp)
            G = [se3_log(Tp)]
            F = [G[0] - se3_log(T_prev)]
            n = 0                                        # k - k_start = n + 1
            capped = True
            while n + 1 <= params.max_iters:
                cnt["iterations"] += 1
                E = energy(Ck, nu)
                if E >= E_prev:                          # safeguard: revert to T'
                    cnt["reverts"] += 1
                    Tk, Ck = Tp, corr(Tp)
                    E = energy(Ck, nu)
                elif n > 0:
                    cnt["aa_accepted"] += 1
                E_prev = E
                trace.append(E)
                Tp = align(Ck, nu)
                if np.linalg.norm(Tk - Tp) < params.eps:   # Frobenius norm of the 4x4 difference
                    capped = False
                    break
                Gk = se3_log(Tp)
                G.append(Gk)
                F.append(Gk - se3_log(Tk))
                mk = min(n + 1, m)
                x_new = Gk
                if mk > 0:
                    dF = np.stack([(F[-j] - F[-j - 1]).ravel() for j in range(1, mk + 1)], 1)
                    theta = anderson_theta(F[-1].ravel(), dF)
                    if theta is not None:
                        x_new = Gk - sum(theta[j - 1] * (G[-j] - G[-j - 1]) for j in range(1, mk + 1))
                Tk = se3_exp(x_new)
                Ck = corr(Tk)
                n += 1
            if capped:
                # Reading: the iterate carried out of a stage on the iteration cap is
                # energy-checked like any other (Sec. 4.2's monotone-decrease safeguard).
                if energy(Ck, nu) >= E_prev:
                    cnt["reverts"] += 1
                    Tk, Ck = Tp, None
            if nu == nu_min:
                break
            nu = max(nu / 2.0, nu_min)
            T_prev = Tk
            C_prev = Ck if Ck is not None else corr(Tk)
    except Degenerate:
        return _result(nz, Tk, cnt, nu_max, nu_min, E_prev, trace, status="degenerate")
    return _result(nz, Tk, cnt, nu_max, nu_min, E_prev, trace)


# ---------------------------------------------------------------------------
# Point-to-plane (Sec. 5, App. D) and Algorithm 2
# ---------------------------------------------------------------------------

def se3_partials(xi: np.ndarray):
    """App. D: R = exp(delta^) and the partial derivatives of R and of the
    translation t(delta, u) = ((R - I) u^ delta + delta delta^T u) / |delta|^2
    with respect to xi = [delta; u]. Returns (R, dR (list of three 3x3),
    dt/d delta (3x3, column j), dt/du (3x3))."""
    delta, u = np.asarray(xi[:3], np.float64), np.asarray(xi[3:6], np.float64)
    th2 = float(delta @ delta)
    th = math.sqrt(th2)
    I = np.eye(3)
    R = sla.expm(hat(delta))
    if th2 == 0.0:
        # App. D special case at delta = 0.
        dR = [hat(I[:, j]) for j in range(3)]
        dt_dd = np.zeros((3, 3))
        dt_du = I.copy()
    elif th < SMALL_DELTA:
        # Reading: second-order series of the same quantities for tiny |delta|.
        Jl = I + 0.5 * hat(delta) + hat(delta) @ hat(delta) / 6.0
        dR = [hat(Jl[:, j]) @ R for j in range(3)]
        dt_dd = np.stack([0.5 * np.cross(I[:, j], u)
                          + (np.cross(I[:, j], np.cross(delta, u)) + np.cross(delta, np.cross(I[:, j], u))) / 6.0
                          for j in range(3)], 1)
        dt_du = Jl
    else:
        dR = [(delta[j] * hat(delta) + hat(np.cross(delta, (I - R)[:, j]))) / th2 @ R for j in range(3)]
        Mm = (R - I) @ hat(u) + float(delta @ u) * I
        D = np.stack([dR[j] @ hat(u) @ delta for j in range(3)], 1)
        # Reading: App. D's last term "M delta^T delta" is the outer product M delta delta^T
        # (the derivative of 1/|delta|^2 times M delta).
        dt_dd = (Mm + np.outer(delta, u) + D) / th2 - 2.0 / (th2 * th2) * Mm @ np.outer(delta, delta)
        dt_du = ((I - R) @ hat(delta) + np.outer(delta, delta)) / th2
    return R, dR, dt_dd, dt_du


def plane_gradient(xi: np.ndarray, P: np.ndarray, Nq: np.ndarray) -> np.ndarray:
    """J_i of Eq. (17) for every source point (App. D). Returns [M, 6].

    B_i(xi) = (R p_i + t - q_i) . n_i, xi = [delta; u], R = exp(delta^),
    t = ((R - I) u^ delta + delta delta^T u) / |delta|^2.
    """
    _, dR, dt_dd, dt_du = se3_partials(xi)
    # dB/dR = n p^T, dB/dt = n (App. D)
    Jd = np.stack([np.einsum("ni,ij,nj->n", Nq, dR[j], P) + Nq @ dt_dd[:, j] for j in range(3)], 1)
    Ju = Nq @ dt_du
    return np.concatenate([Jd, Ju], axis=1)


def symmetric_residual(xi: np.ndarray, P: np.ndarray, Qh: np.ndarray, Nq: np.ndarray, Np: np.ndarray):
    """Residual of the symmetric objective (the extension Sec. 7 proposes):
    H_i(xi) = (R p_i + t - q_i) . (R np_i + nq_i), the sum of the two surfaces'
    normals at the pair, the source normal carried by the motion. Returns
    (H [M], X = R p + t [M,3], the summed normals [M,3])."""
    T = se3_transform(xi)
    X = apply(T, P)
    Ns = Np @ T[:3, :3].T + Nq
    return np.einsum("nd,nd->n", X - Qh, Ns), X, Ns


def symmetric_gradient(xi: np.ndarray, P: np.ndarray, Qh: np.ndarray, Nq: np.ndarray, Np: np.ndarray) -> np.ndarray:
    """dH_i / dxi of symmetric_residual for every source point, from App. D's
    partials: d H / d delta_j = (dR_j p + dt/d delta_j) . (R np + nq)
    + (R p + t - q) . (dR_j np), d H / d u = (dt/du)^T (R np + nq). Returns [M, 6]."""
    _, dR, dt_dd, dt_du = se3_partials(xi)
    _, X, Ns = symmetric_residual(xi, P, Qh, Nq, Np)
    Dv = X - Qh
    Jd = np.stack([np.einsum("ni,ij,nj->n", Ns, dR[j], P) + Ns @ dt_dd[:, j]
                   + np.einsum("ni,ij,nj->n", Dv, dR[j], Np) for j in range(3)], 1)
    Ju = Ns @ dt_du
    return np.concatenate([Jd, Ju], axis=1)


def se3_transform(xi) -> np.ndarray:
    return se3_exp(se3_matrix(xi))


def register_point_to_plane(P32, Q32, N32, params: Params, T0=None, Np32=None) -> dict:
    """Algorithm 2 (Welsch point-to-plane ICP with AA). params.variant 'p2pl'
    runs the plain point-to-plane objective of Eq. (15) the same way. Reading:
    psi(x) = x^2, so gamma_i = 1 and the energy is sum H_i^2, and a single stage
    whose iteration cap is max_iters (the caps 6..10 of Sec. 5 belong to the nu
    stages, which plain point-to-plane does not have).

    params.variant 'sym_welsch' (source normals Np32 required) runs the robust
    symmetric objective Sec. 7 proposes as future work, read as Alg. 2 with the
    residual H_i of symmetric_residual in place of Eq. (15)'s: Welsch weights and
    energy on H_i, the Gauss-Newton system of Eq. (18) with its gradient
    symmetric_gradient, the same Anderson step, line search and nu stages, and
    nu_min from the target's statistic of Sec. 5."""
    sym = params.variant == "sym_welsch"
    robust = params.variant in ("p2pl_welsch", "sym_welsch")
    P = np.asarray(P32, dtype=np.float64)
    Q = np.asarray(Q32, dtype=np.float64)
    Nr = np.asarray(N32, dtype=np.float64)       # normals used as given
    Np = np.asarray(Np32, dtype=np.float64) if sym else None
    nz = normalization(P, Q)
    Pn, Qn = nz.fwd(P), nz.fwd(Q)
    cnt = _counters()
    trace = []
    m = params.anderson_m

    nn = nn_function(Qn, params.nn)

    def evaluate(xi, nu):
        """One correspondence pass at xi: closest points, B_i and the energy."""
        cnt["corr_passes"] += 1
        T = se3_transform(xi)
        idx, _, _ = nn(apply(T, Pn))
        n = Nr[idx]
        if sym:
            B, _, _ = symmetric_residual(xi, Pn, Qn[idx], n, Np)
        else:
            B = np.einsum("nd,nd->n", apply(T, Pn) - Qn[idx], n)
        if robust:
            E = float(welsch(B, nu).sum()) if nu is not None else None
        else:
            E = float((B * B).sum())
        return dict(xi=np.array(xi, dtype=np.float64), idx=idx, B=B, n=n, E=E, Qh=Qn[idx])

    _, jit_xi = _jitter(params)

    def gn_map(ev, nu):
        """G_ppl (Eq. 19): solve the Gauss-Newton system of Eq. (18) at ev['xi'].

        Reading: the right-hand side is sum_i gamma_i J_i (J_i^T xi_k - B_i), the
        stationarity condition of the linearised Eq. (16); the printed sign of
        B_i - J_i^T xi_k maps a true fixed point away from itself.
        """
        xi = ev["xi"]
        gamma = np.exp(-ev["B"] ** 2 / (2.0 * nu * nu)) if robust else np.ones_like(ev["B"])
        J = symmetric_gradient(xi, Pn, ev["Qh"], ev["n"], Np) if sym else plane_gradient(xi, Pn, ev["n"])
        A = (J * gamma[:, None]).T @ J
        b = (J * gamma[:, None]).T @ (J @ xi - ev["B"])
        # Reading for points in a plane (Sec. 3: the problem is stated in R^d):
        # embedded at z = 0 with in-plane normals, the directions that tilt the
        # plane or move along z change no distance, so their rows, columns and
        # right-hand sides are exactly zero; they keep a zero step and the rest
        # is the 2-D system. 3-D data has no such direction.
        act = ~((A == 0.0).all(axis=1) & (A == 0.0).all(axis=0) & (b == 0.0))
        if not act.any():
            raise Degenerate("singular point-to-plane system")
        x = np.zeros(6)
        try:
            cf = sla.cho_factor(A[np.ix_(act, act)])
        except np.linalg.LinAlgError as e:
            raise Degenerate("singular point-to-plane system") from e
        x[act] = sla.cho_solve(cf, b[act])
        return jit_xi(x)

    xi0 = np.zeros(6) if T0 is None else se3_vee(se3_log(nz.T_to_normalized(np.asarray(T0, np.float64))))
    ev_prev = evaluate(xi0, None)
    if robust:
        nu_max = params.nu_max if params.nu_max > 0 else 3.0 * float(np.median(np.abs(ev_prev["B"])))
        nu_min = params.nu_min if params.nu_min > 0 else nu_min_point_to_plane(Qn, Nr)
        nu_min = max(nu_min, params.nu_min_floor)
        nu_max = max(nu_max, nu_min)
        cap = params.p2pl_iters_first
    else:                                             # one stage (nu unused)
        nu_max = nu_min = 1.0
        cap = params.max_iters
    nu = nu_max
    x_prev = xi0
    xk = xi0
    E_prev = math.inf

    def line_search(x_from, x_star, ev_k, E_prev):
        """Alg. 2: search along x_star - x_from, keeping the lowest energy seen."""
        best = ev_k
        tau = 1.0
        for _ in range(params.max_line_search):
            ev_t = evaluate(x_from + tau * (x_star - x_from), nu)
            cnt["line_search_trials"] += 1
            if ev_t["E"] < best["E"]:
                best = ev_t
            if ev_t["E"] < E_prev:
                break
            tau *= 0.5
        return best

    try:
        while True:
            cnt["stages"] += 1
            E_prev = math.inf
            x_star = gn_map(ev_prev, nu)                  # xi*^(k) = G(xi^(k-1))
            xk = x_star
            G = [x_star]
            F = [x_star - x_prev]
            n = 0
            capped = True
            ev_last = None
            while n + 1 <= cap:
                cnt["iterations"] += 1
                ev = evaluate(xk, nu)
                if ev["E"] >= E_prev:
                    cnt["reverts"] += 1
                    ev = line_search(x_prev, x_star, ev, E_prev)
                    xk = ev["xi"]
                elif n > 0:
                    cnt["aa_accepted"] += 1
                E_prev = ev["E"]
                trace.append(E_prev)
                x_star_next = gn_map(ev, nu)              # xi*^(k+1) = G(xi^(k))
                if np.linalg.norm(x_star_next - xk) < params.eps:
                    capped = False
                    ev_last = ev
                    break
                Gk = x_star_next
                G.append(Gk)
                F.append(Gk - xk)
                mk = min(n + 1, m)
                x_new = Gk
                if mk > 0:
                    dF = np.stack([F[-j] - F[-j - 1] for j in range(1, mk + 1)], 1)
                    theta = anderson_theta(F[-1], dF)
                    if theta is not None:
                        # Reading: no exp here; xi is already the parameter vector.
                        x_new = Gk - sum(theta[j - 1] * (G[-j] - G[-j - 1]) for j in range(1, mk + 1))
                x_prev, x_star, xk = xk, x_star_next, x_new
                n += 1
            if capped:
                # Reading: the iterate carried out on the cap gets the same check.
                ev = evaluate(xk, nu)
                if ev["E"] >= E_prev:
                    cnt["reverts"] += 1
                    ev = line_search(x_prev, x_star, ev, E_prev)
                    xk = ev["xi"]
                ev_last = ev
            if nu == nu_min:
                break
            nu = max(nu / 2.0, nu_min)
            cap = min(cap + 1, params.p2pl_iters_cap)   # robust only: plain has one stage
            x_prev = xk
            ev_prev = ev_last
    except Degenerate:
        return _result(nz, se3_transform(xk), cnt, nu_max, nu_min, E_prev, trace, status="degenerate")
    return _result(nz, se3_transform(xk), cnt, nu_max, nu_min, E_prev, trace)


def register(P32, Q32, params: Params, normals=None, T0=None, source_normals=None) -> dict:
    if params.variant in ("p2p", "p2p_welsch"):
        return register_point_to_point(P32, Q32, params, T0)
    if params.variant in ("p2pl_welsch", "p2pl", "sym_welsch"):
        if normals is None:
            raise ValueError("point-to-plane needs target normals")
        if params.variant == "sym_welsch" and source_normals is None:
            raise ValueError("the symmetric objective needs source normals")
        return register_point_to_plane(P32, Q32, normals, params, T0, source_normals)
    raise ValueError(params.variant)


def rmse(P32, R, t, R_gt, t_gt) -> float:
    """Eq. (13): RMSE between the computed and the ground-truth motion of P."""
    P = np.asarray(P32, dtype=np.float64)
    d = P @ (R_gt - R).T + (t_gt - t)
    return float(np.sqrt((d * d).sum(axis=1).mean()))
