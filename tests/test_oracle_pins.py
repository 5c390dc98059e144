"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names the passage of the paper it pins and the independent reference:
a library routine computing the same definition, a closed form, an invariant
the paper proves, or brute force on tiny inputs.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.spatial.transform import Rotation

import oracle


def _rot(g, max_angle=math.pi * 0.9):
    axis = g.standard_normal(3)
    axis /= np.linalg.norm(axis)
    return Rotation.from_rotvec(axis * max_angle * g.random()).as_matrix()


# --------------------------------------------------------------------------
# Correspondence step (Sec. 3 Eq. 3): brute force is the definition.
# --------------------------------------------------------------------------

def test_closest_matches_dense_argmin_with_ties():
    g = np.random.default_rng(1)
    Q = g.random((57, 3))
    Q[30] = Q[7]                      # duplicate target: tie must go to index 7
    Q[44] = Q[7]
    X = np.concatenate([g.random((40, 3)), Q[[7, 12]] + 0.0])
    idx, d2, d2s = oracle.closest(X, Q)
    D = ((X[:, None, :] - Q[None]) ** 2).sum(-1)
    assert np.array_equal(idx, D.argmin(1))        # numpy argmin: first minimum
    assert np.allclose(d2, D.min(1), rtol=0, atol=1e-15)
    Ds = np.sort(D, 1)
    assert np.allclose(d2s, Ds[:, 1], rtol=0, atol=1e-15)
    assert idx[40] == 7 and d2[40] == 0.0 and d2s[40] == 0.0


def test_knn_self_matches_stable_sort():
    g = np.random.default_rng(2)
    Q = g.random((80, 3))
    Q[10] = Q[3]                      # duplicates at distance 0 count
    idx, d2 = oracle.knn_self(Q, 6)
    D = ((Q[:, None, :] - Q[None]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    ref = np.argsort(D, axis=1, kind="stable")[:, :6]
    assert np.array_equal(idx, ref)
    assert np.allclose(d2, np.take_along_axis(D, ref, 1), rtol=0, atol=1e-15)
    assert idx[3, 0] == 10 and d2[3, 0] == 0.0


# --------------------------------------------------------------------------
# Alignment step (Eq. 4 and Eq. 12): weighted Procrustes.
# --------------------------------------------------------------------------

def test_procrustes_recovers_known_motion_exactly():
    g = np.random.default_rng(3)
    for _ in range(20):
        P = g.standard_normal((30, 3))
        R, t = _rot(g), g.standard_normal(3)
        w = g.random(30) + 0.01
        T = oracle.weighted_procrustes(P, P @ R.T + t, w)
        assert np.abs(T[:3, :3] - R).max() < 1e-12
        assert np.abs(T[:3, 3] - t).max() < 1e-12


def test_procrustes_beats_dense_rotation_search():
    """The closed form must be at least as good as any rotation on a dense grid."""
    g = np.random.default_rng(4)
    P = g.standard_normal((6, 3))
    Qh = g.standard_normal((6, 3))
    w = g.random(6)
    T = oracle.weighted_procrustes(P, Qh, w)

    def cost(R):
        pbar = (w[:, None] * P).sum(0) / w.sum()
        qbar = (w[:, None] * Qh).sum(0) / w.sum()
        r = P @ R.T + (qbar - R @ pbar) - Qh
        return float((w * (r * r).sum(1)).sum())

    c_closed = cost(T[:3, :3])
    rots = Rotation.random(40000, random_state=5).as_matrix()
    costs = np.array([cost(R) for R in rots])
    best = rots[costs.argmin()]
    assert c_closed <= costs.min() + 1e-12
    # local refinement of the sampled best lands on the closed form
    x = Rotation.from_matrix(best).as_rotvec()
    for step in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        for _ in range(200):
            moved = False
            for d in np.concatenate([np.eye(3), -np.eye(3)]) * step:
                c_new = cost(Rotation.from_rotvec(x + d).as_matrix())
                if c_new < cost(Rotation.from_rotvec(x).as_matrix()):
                    x, moved = x + d, True
            if not moved:
                break
    assert abs(cost(Rotation.from_rotvec(x).as_matrix()) - c_closed) < 1e-9
    # and a translation check: t = qbar - R pbar is optimal given R
    assert np.linalg.det(T[:3, :3]) == pytest.approx(1.0, abs=1e-12)


def test_procrustes_rejects_zero_weights():
    with pytest.raises(oracle.Degenerate):
        oracle.weighted_procrustes(np.ones((3, 3)), np.ones((3, 3)), np.zeros(3))


# --------------------------------------------------------------------------
# SE(3) exp / log (Eqs. 8-9, App. A).
# --------------------------------------------------------------------------

def _rodrigues_se3(xi):
    """Textbook closed form: R = I + sin K + (1-cos) K^2, t = V u (Gallier & Xu)."""
    w, u = xi[:3], xi[3:]
    th = np.linalg.norm(w)
    K = oracle.hat(w / th)
    R = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    V = np.eye(3) + (1 - math.cos(th)) / th * K + (th - math.sin(th)) / th * K @ K
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ u
    return T


def test_exp_matches_rodrigues_closed_form():
    g = np.random.default_rng(6)
    for _ in range(50):
        xi = np.concatenate([_rot_vec(g), g.standard_normal(3)])
        T = oracle.se3_exp(oracle.se3_matrix(xi))
        assert np.abs(T - _rodrigues_se3(xi)).max() < 1e-13


def _rot_vec(g, max_angle=3.0):
    a = g.standard_normal(3)
    return a / np.linalg.norm(a) * max_angle * g.random()


def _log_by_schur(T):
    """App. A's construction, written from the appendix with scipy's real Schur form.

    R = Q1 D Q1^T with D = diag(D_1, 1); log(U') = [[B, V y], [0, 0]] with
    B = theta * [[0,-1],[1,0]] on the 2x2 block, y = Q1^T t and
    V = I - theta/2 K + (1 - theta sin / (2 (1 - cos))) K^2, K the unit generator.
    """
    R, t = T[:3, :3], T[:3, 3]
    D, Q1 = sla.schur(R, output="real")
    # put the 2x2 rotation block first
    if abs(D[2, 1]) > abs(D[1, 0]):
        perm = [1, 2, 0]
        Q1 = Q1[:, perm]
        D = Q1.T @ R @ Q1
    th = math.atan2(D[1, 0] - D[0, 1], D[0, 0] + D[1, 1])
    K = np.zeros((3, 3))
    K[0, 1], K[1, 0] = -1.0, 1.0
    c = 1 - th * math.sin(th) / (2 * (1 - math.cos(th)))
    V = np.eye(3) - th / 2 * K + c * K @ K
    L = np.zeros((4, 4))
    L[:3, :3] = Q1 @ (th * K) @ Q1.T
    L[:3, 3] = Q1 @ (V @ (Q1.T @ t))
    return L


def test_log_matches_appendix_a_schur_construction():
    g = np.random.default_rng(7)
    for _ in range(50):
        xi = np.concatenate([_rot_vec(g, 3.0) + 1e-3, g.standard_normal(3)])
        T = oracle.se3_exp(oracle.se3_matrix(xi))
        L = oracle.se3_log(T)
        assert np.abs(L - _log_by_schur(T)).max() < 1e-10
        assert np.abs(oracle.se3_vee(L) - xi).max() < 1e-10      # principal branch, angle < pi
        assert np.abs(oracle.se3_exp(L) - T).max() < 1e-13


def test_log_small_and_zero_angle():
    T = np.eye(4)
    T[:3, 3] = [0.3, -0.2, 0.1]
    assert np.abs(oracle.se3_log(T)[:3, 3] - T[:3, 3]).max() < 1e-15
    xi = np.array([1e-9, -2e-9, 3e-9, 0.1, 0.2, 0.3])
    L = oracle.se3_log(oracle.se3_exp(oracle.se3_matrix(xi)))
    assert np.abs(oracle.se3_vee(L) - xi).max() < 1e-15


# --------------------------------------------------------------------------
# App. D gradient: translation formula and central finite differences.
# --------------------------------------------------------------------------

def test_appendix_d_translation_formula_equals_exp():
    g = np.random.default_rng(8)
    for _ in range(20):
        d, u = _rot_vec(g), g.standard_normal(3)
        T = oracle.se3_exp(oracle.se3_matrix(np.concatenate([d, u])))
        R = T[:3, :3]
        t = ((R - np.eye(3)) @ oracle.hat(u) @ d + np.outer(d, d) @ u) / (d @ d)
        assert np.abs(t - T[:3, 3]).max() < 1e-13


def _B(xi, P, Qh, Nq):
    T = oracle.se3_transform(xi)
    return np.einsum("nd,nd->n", oracle.apply(T, P) - Qh, Nq)


@pytest.mark.parametrize("delta_scale", [1.0, 0.3, 1e-3, 1e-7, 0.0])
def test_plane_gradient_central_differences(delta_scale):
    g = np.random.default_rng(9)
    P = g.standard_normal((12, 3))
    Qh = g.standard_normal((12, 3))
    Nq = g.standard_normal((12, 3))
    Nq /= np.linalg.norm(Nq, axis=1, keepdims=True)
    d = _rot_vec(g, 2.0)
    d = d / np.linalg.norm(d) * delta_scale if delta_scale else np.zeros(3)
    u = g.standard_normal(3) if delta_scale else np.zeros(3)   # App. D's delta=0 case is exact at u=0
    xi = np.concatenate([d, u])
    J = oracle.plane_gradient(xi, P, Nq)
    h = 1e-6
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        fd = (_B(xi + e, P, Qh, Nq) - _B(xi - e, P, Qh, Nq)) / (2 * h)
        assert np.abs(J[:, j] - fd).max() < 1e-7 * max(1.0, np.abs(fd).max()), (j, delta_scale)


# --------------------------------------------------------------------------
# Point-to-plane Gauss-Newton sign (Eq. 18): the true motion is a fixed point.
# --------------------------------------------------------------------------

def test_gauss_newton_fixed_point_and_printed_sign():
    g = np.random.default_rng(10)
    Q = g.standard_normal((200, 3))
    Nq = g.standard_normal((200, 3))
    Nq /= np.linalg.norm(Nq, axis=1, keepdims=True)
    xi_true = np.concatenate([_rot_vec(g, 0.5), 0.3 * g.standard_normal(3)])
    T = oracle.se3_transform(xi_true)
    P = (Q - T[:3, 3]) @ T[:3, :3]            # R p + t = q exactly
    B = _B(xi_true, P, Q, Nq)
    assert np.abs(B).max() < 1e-12
    J = oracle.plane_gradient(xi_true, P, Nq)
    A = J.T @ J
    x_read = np.linalg.solve(A, J.T @ (J @ xi_true - B))      # the reading
    x_printed = np.linalg.solve(A, J.T @ (B - J @ xi_true))   # as printed
    assert np.abs(x_read - xi_true).max() < 1e-10
    assert np.abs(x_printed + xi_true).max() < 1e-10           # lands on -xi


# --------------------------------------------------------------------------
# Anderson acceleration (Eq. 6).
# --------------------------------------------------------------------------

def test_anderson_lstsq_matches_numpy():
    g = np.random.default_rng(11)
    for mk in range(1, 6):
        dF = g.standard_normal((16, mk))
        F = g.standard_normal(16)
        th = oracle.anderson_theta(F, dF)
        ref = np.linalg.lstsq(dF, F, rcond=None)[0]
        assert np.abs(th - ref).max() < 1e-12


def test_anderson_rank_rule():
    dF = np.ones((6, 2))
    assert oracle.anderson_theta(np.ones(6), dF) is None
    assert oracle.anderson_theta(np.ones(6), np.zeros((6, 1))) is None


def test_anderson_solves_linear_fixed_point_in_dim_plus_one_steps():
    """AA with m >= dim on G(x) = A x + b terminates (GMRES equivalence, Walker & Ni 2011)."""
    g = np.random.default_rng(12)
    n = 4
    A = 0.5 * g.standard_normal((n, n)) / math.sqrt(n)
    b = g.standard_normal(n)
    x_star = np.linalg.solve(np.eye(n) - A, b)
    G = lambda x: A @ x + b
    x = np.zeros(n)
    Gs, Fs = [G(x)], [G(x) - x]
    x = Gs[0]
    for k in range(1, n + 2):
        Gk = G(x)
        Gs.append(Gk)
        Fs.append(Gk - x)
        mk = min(k, n)
        dF = np.stack([Fs[-j] - Fs[-j - 1] for j in range(1, mk + 1)], 1)
        th = oracle.anderson_theta(Fs[-1], dF)
        x = Gk - sum(th[j - 1] * (Gs[-j] - Gs[-j - 1]) for j in range(1, mk + 1))
    assert np.abs(x - x_star).max() < 1e-9


# --------------------------------------------------------------------------
# Welsch surrogate (Eq. 11, App. B).
# --------------------------------------------------------------------------

def test_welsch_surrogate_majorizes():
    g = np.random.default_rng(13)
    x = 3 * g.random(10000)
    y = 3 * g.random(10000)
    nu = 0.2 + g.random()
    assert np.all(oracle.welsch_surrogate(x, y, nu) >= oracle.welsch(x, nu) - 1e-15)
    assert np.abs(oracle.welsch_surrogate(y, y, nu) - oracle.welsch(y, nu)).max() < 1e-15
    assert np.all(oracle.welsch(x, nu) < 1.0) and np.all(oracle.welsch(x, nu) >= 0.0)


# --------------------------------------------------------------------------
# Scale of Welsch's function (Eq. 10) fixed by App. C: nu_min is chosen by the
# three-sigma rule, so nu is the standard deviation of the Gaussian weight
# exp(-x^2 / (2 nu^2)) that Eq. 11 / Eq. 12 put on each residual. At one sigma
# the weight is e^(-1/2); at three sigma e^(-9/2) (an outlier beyond 3 nu has
# almost no weight, psi almost 1). A slip of nu^2 for 2 nu^2 (or the reverse)
# gives e^(-1) and e^(-9), or e^(-1/4) and e^(-9/4).
# --------------------------------------------------------------------------

SIGMA1_W, SIGMA3_W = math.exp(-0.5), math.exp(-4.5)


def test_welsch_function_is_one_minus_a_gaussian_of_sigma_nu():
    for nu in (1e-3, 0.37, 5.0):
        assert oracle.welsch(nu, nu) == pytest.approx(1.0 - SIGMA1_W, rel=1e-14)
        assert oracle.welsch(3.0 * nu, nu) == pytest.approx(1.0 - SIGMA3_W, rel=1e-14)
        assert oracle.welsch(-2.0 * nu, nu) == pytest.approx(1.0 - math.exp(-2.0), rel=1e-14)
        assert oracle.welsch(0.0, nu) == 0.0
    # three-sigma rule: a residual beyond 3 nu is treated as an outlier, psi > 0.98
    assert oracle.welsch(3.0, 1.0) > 0.98


def _two_height_pair(nu_n):
    """A 10 x 10 grid of spacing 1 in the plane z = 0 (normals +z) and the same
    grid lifted by heights that are nu and 3 nu in normalised units, in a
    checkerboard. The closest point of each lifted point is the one below it
    (heights < 1). Returns P, Q, normals and the lifted heights in normalised
    units."""
    gx = np.arange(10, dtype=np.float64)
    X, Y = np.meshgrid(gx, gx)
    Q = np.stack([X.ravel(), Y.ravel(), np.zeros(100)], 1)
    lift = np.where((X.ravel() + Y.ravel()) % 2 == 0, 1.0, 3.0)
    # the bounding-box diagonal of P u Q includes the largest lift: solve for it
    diag = math.sqrt(2 * 81.0 / (1.0 - 9.0 * nu_n * nu_n))
    P = Q.copy()
    P[:, 2] = lift * nu_n * diag
    P32, Q32 = P.astype(np.float32), Q.astype(np.float32)
    nz = oracle.normalization(P32.astype(np.float64), Q32.astype(np.float64))
    heights = nz.s * (P32[:, 2].astype(np.float64) - nz.c[2])
    N = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (100, 1))
    return P32, Q32, N, lift, heights


def test_weights_inside_algorithm_1_are_gaussian_of_sigma_nu(monkeypatch):
    """The weights Alg. 1's alignment step (Eq. 12) receives at the start,
    captured from the registration itself: e^(-1/2) at one sigma, e^(-9/2) at
    three sigma."""
    nu_n = 0.02
    P, Q, _, lift, heights = _two_height_pair(nu_n)
    assert np.allclose(heights, lift * nu_n, rtol=1e-6)
    seen = []
    real = oracle.weighted_procrustes

    def spy(Pn, Qh, w):
        seen.append(np.array(w))
        return real(Pn, Qh, w)

    monkeypatch.setattr(oracle, "weighted_procrustes", spy)
    oracle.register(P, Q, oracle.Params(variant="p2p_welsch", nu_max=nu_n, nu_min=nu_n, max_iters=2))
    w0 = seen[0]
    assert np.allclose(w0[lift == 1.0], SIGMA1_W, rtol=1e-5)
    assert np.allclose(w0[lift == 3.0], SIGMA3_W, rtol=1e-5)


def test_weights_inside_algorithm_2_are_gaussian_of_sigma_nu(monkeypatch):
    """The Gauss-Newton system of Eq. 18 that Alg. 2 factors at the start
    (identity, normals +z): its u_z diagonal is sum gamma_i and its right-hand
    side -sum gamma_i B_i, with gamma_i e^(-1/2) at one sigma and e^(-9/2) at
    three sigma."""
    nu_n = 0.02
    P, Q, N, lift, heights = _two_height_pair(nu_n)
    seen = []

    class SlaSpy:
        def __getattr__(self, name):
            return getattr(sla, name)

        def cho_factor(self, A, *a, **k):
            seen.append(("A", np.array(A)))
            return sla.cho_factor(A, *a, **k)

        def cho_solve(self, cf, b, *a, **k):
            seen.append(("b", np.array(b)))
            return sla.cho_solve(cf, b, *a, **k)

    monkeypatch.setattr(oracle, "sla", SlaSpy())
    oracle.register(P, Q, oracle.Params(variant="p2pl_welsch", nu_max=nu_n, nu_min=nu_n), normals=N)
    A = next(v for k, v in seen if k == "A")
    b = next(v for k, v in seen if k == "b")
    # planar target: delta_z, u_x and u_y change no distance, so the system is the
    # (delta_x, delta_y, u_z) block, u_z last
    assert A.shape == (3, 3)
    n1, n3 = int((lift == 1.0).sum()), int((lift == 3.0).sum())
    assert A[2, 2] == pytest.approx(n1 * SIGMA1_W + n3 * SIGMA3_W, rel=1e-5)
    assert -b[2] == pytest.approx(nu_n * (n1 * SIGMA1_W + 3.0 * n3 * SIGMA3_W), rel=1e-5)


# --------------------------------------------------------------------------
# nu_min rationale (App. C): a planar square grid of spacing h gives E_Q = h.
# --------------------------------------------------------------------------

def test_nu_min_square_grid():
    h = 0.01
    gx = np.arange(40) * h
    X, Y = np.meshgrid(gx, gx)
    Q = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    assert oracle.nu_min_point_to_point(Q) == pytest.approx(h / (3 * math.sqrt(3)), rel=1e-12)
    N = np.tile([0.0, 0.0, 1.0], (Q.shape[0], 1))
    assert oracle.nu_min_point_to_plane(Q, N) == 0.0


# --------------------------------------------------------------------------
# Whole algorithms: MM monotonicity, safeguard, exact recovery.
# --------------------------------------------------------------------------

def _surface_pair(seed, n=600, angle=0.3, noise=0.0):
    g = np.random.default_rng(seed)
    xy = g.random((n, 2))
    z = 0.2 * np.sin(3 * xy[:, 0]) * np.cos(2 * xy[:, 1]) + 0.1 * xy[:, 0] ** 2
    Q = np.stack([xy[:, 0], xy[:, 1], z], 1)
    gz = np.stack([-0.6 * np.cos(3 * xy[:, 0]) * np.cos(2 * xy[:, 1]) - 0.2 * xy[:, 0],
                   0.4 * np.sin(3 * xy[:, 0]) * np.sin(2 * xy[:, 1]), np.ones(n)], 1)
    N = gz / np.linalg.norm(gz, axis=1, keepdims=True)
    R = Rotation.from_rotvec(angle * np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])).as_matrix()
    t = np.array([0.05, -0.03, 0.02])
    P = (Q - t) @ R + noise * g.standard_normal(Q.shape)     # R p + t = q
    return P.astype(np.float32), Q.astype(np.float32), N.astype(np.float32), R, t


@pytest.mark.parametrize("variant", ["p2p", "p2p_welsch"])
def test_plain_mm_energy_is_monotone(variant):
    P, Q, _, _, _ = _surface_pair(14, n=500, angle=0.2, noise=0.002)
    g = np.random.default_rng(14)
    Qo = np.concatenate([Q, (g.random((100, 3)) * [1, 1, 0.3]).astype(np.float32)])
    prm = oracle.Params(variant=variant, anderson_m=0, max_iters=60,
                        nu_max=0.05 if variant == "p2p_welsch" else 0,
                        nu_min=0.05 if variant == "p2p_welsch" else 0)
    r = oracle.register(P, Qo, prm)
    tr = r["trace"]
    assert len(tr) > 3
    assert np.all(np.diff(tr) <= 1e-12 * np.abs(tr[:-1]))


def test_safeguard_keeps_accepted_energy_monotone():
    P, Q, N, _, _ = _surface_pair(15, n=500, angle=0.3, noise=0.003)
    r = oracle.register(P, Q, oracle.Params(variant="p2p", max_iters=100))
    assert np.all(np.diff(r["trace"]) <= 0.0)
    # plain point-to-plane: one stage, the line search keeps the accepted energy monotone too
    r = oracle.register(P, Q, oracle.Params(variant="p2pl", max_iters=100), normals=N)
    assert r["stages"] == 1 and np.all(np.diff(r["trace"]) <= 0.0)


def test_plain_point_to_plane_has_one_stage_capped_by_max_iters():
    P, Q, N, _, _ = _surface_pair(19, n=400, angle=0.2, noise=0.004)
    r = oracle.register(P, Q, oracle.Params(variant="p2pl", max_iters=3), normals=N)
    assert r["stages"] == 1 and r["iterations"] <= 3
    assert r["nu_max"] == 1.0 and r["nu_min"] == 1.0


def test_safeguard_reverts_bad_anderson_steps(monkeypatch):
    """With every AA step sabotaged, Alg. 1 reduces to plain MM plus one revert per step."""
    P, Q, _, _, _ = _surface_pair(16, n=400, angle=0.25, noise=0.002)
    plain = oracle.register(P, Q, oracle.Params(variant="p2p", anderson_m=0, max_iters=200))
    monkeypatch.setattr(oracle, "anderson_theta", lambda F, dF: np.full(dF.shape[1], 50.0))
    bad = oracle.register(P, Q, oracle.Params(variant="p2p", anderson_m=5, max_iters=200))
    assert bad["iterations"] == plain["iterations"]
    assert bad["reverts"] == bad["iterations"] - 1 - plain["reverts"]
    assert bad["aa_accepted"] == 0
    assert np.abs(bad["R"] - plain["R"]).max() < 1e-12
    # plain MM moves to exp(log T'), the revert to T' itself: equal up to rounding
    assert np.allclose(bad["trace"], plain["trace"], rtol=1e-10, atol=0)


@pytest.mark.parametrize("variant", ["p2p", "p2p_welsch", "p2pl_welsch", "p2pl"])
def test_exact_copy_is_recovered(variant):
    P, Q, N, R, t = _surface_pair(17, n=800, angle=0.15)
    r = oracle.register(P, Q, oracle.Params(variant=variant), normals=N)
    assert r["status"] == "ok"
    # float32 inputs: the copy is exact only to float32 rounding
    assert np.abs(r["R"] - R).max() < 1e-5
    assert np.abs(r["t"] - t).max() < 1e-5
    if variant in ("p2p", "p2pl"):
        assert r["final_energy"] < 1e-9


def test_normalization_round_trip():
    g = np.random.default_rng(18)
    P, Q = g.random((20, 3)) * 5 + 3, g.random((30, 3)) * 4 - 1
    nz = oracle.normalization(P, Q)
    T = np.eye(4)
    T[:3, :3] = _rot(g)
    T[:3, 3] = g.standard_normal(3)
    Tn = nz.T_to_normalized(T)
    assert np.abs(nz.T_to_original(Tn) - T).max() < 1e-12
    assert np.abs(oracle.apply(Tn, nz.fwd(P)) - nz.fwd(oracle.apply(T, P))).max() < 1e-12
    both = np.concatenate([nz.fwd(P), nz.fwd(Q)])
    assert np.linalg.norm(both.max(0) - both.min(0)) == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("variant", ["p2p", "p2p_welsch", "p2pl_welsch"])
def test_solve_jitter_is_off_by_default_and_small_on_a_well_posed_case(variant):
    """The sensitivity probe leaves the oracle unchanged at 0, and on a
    well-conditioned exact copy a 1e-13 perturbation of every alignment solve
    moves the answer by rounding-level amounts only (so a large spread under it
    is a property of the input, not of the probe)."""
    import dataclasses
    P, Q, N, R, t = _surface_pair(19, n=600, angle=0.1)
    prm = oracle.Params(variant=variant)
    a = oracle.register(P, Q, prm, normals=N)
    b = oracle.register(P, Q, dataclasses.replace(prm, solve_jitter=0.0, jitter_seed=5), normals=N)
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["t"], b["t"])
    assert a["iterations"] == b["iterations"]
    c = oracle.register(P, Q, dataclasses.replace(prm, solve_jitter=1e-13, jitter_seed=5), normals=N)
    assert np.abs(c["R"] - a["R"]).max() < 1e-10
    assert np.abs(c["t"] - a["t"]).max() < 1e-10


# --------------------------------------------------------------------------
# Normal estimate (Sec. 6: PCA over the k nearest neighbours)
# --------------------------------------------------------------------------

def test_knn_all_includes_self_and_orders_by_distance_then_index():
    g = np.random.default_rng(31)
    Q = g.random((400, 3))
    Q[300:310] = Q[5]                                  # duplicates at distance 0
    idx, d2 = oracle.knn_all(Q, 12)
    D = ((Q[:, None, :] - Q[None, :, :]) ** 2).sum(-1)
    for i in range(0, 400, 7):
        order = np.lexsort((np.arange(400), D[i]))[:12]
        assert list(idx[i]) == list(order)
        assert np.array_equal(d2[i], D[i][order])
    assert idx[5, 0] == 5 and set(idx[5, 1:11]) == set(range(300, 310))


def test_normals_of_a_plane_are_its_normal():
    g = np.random.default_rng(32)
    a, b, c = 0.3, -0.7, 0.2
    xy = g.random((3000, 2))
    Q = np.column_stack([xy, a * xy[:, 0] + b * xy[:, 1] + c])
    n_true = np.array([-a, -b, 1.0]) / np.linalg.norm([-a, -b, 1.0])
    v = np.array([0.5, 0.5, 5.0])                      # above the plane
    N = oracle.estimate_normals(Q, 30, viewpoint=v)
    assert np.abs(N - n_true[None, :]).max() < 1e-9
    assert (np.einsum("nd,nd->n", N, v - Q) >= 0).all()


def test_normals_of_a_sphere_are_radial_and_turned_to_the_viewpoint():
    g = np.random.default_rng(33)
    u = g.standard_normal((5000, 3))
    Q = u / np.linalg.norm(u, axis=1, keepdims=True)
    N = oracle.estimate_normals(Q, 30)                 # viewpoint: the origin, inside the sphere
    cos = np.einsum("nd,nd->n", N, -Q)                 # inward
    assert (cos > 0).all()
    ang = np.arccos(np.clip(cos, -1, 1))
    # neighbourhood radius about 0.15: a tilted PCA plane stays within a few degrees
    assert ang.mean() < 0.02 and ang.max() < 0.1


def test_normal_minimises_the_rayleigh_quotient():
    """The normal is the direction of least spread of the neighbourhood: its
    quotient n^T C n is below that of 20000 random unit directions."""
    g = np.random.default_rng(34)
    Q = g.standard_normal((200, 3)) * [1.0, 0.5, 0.1]
    N = oracle.estimate_normals(Q, 30)
    idx, _ = oracle.knn_all(Q, 30)
    U = g.standard_normal((20000, 3))
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    for i in range(0, 200, 17):
        nb = Q[idx[i]]
        C = (nb - nb.mean(0)).T @ (nb - nb.mean(0)) / 30
        qn = N[i] @ C @ N[i]
        assert qn <= np.einsum("nd,de,ne->n", U, C, U).min() + 1e-12
        assert abs(np.linalg.norm(N[i]) - 1.0) < 1e-12


def test_normals_at_sampled_rows_equal_the_full_estimate():
    g = np.random.default_rng(35)
    Q = g.random((1500, 3)) * [1.0, 1.0, 0.05]
    rows = np.arange(0, 1500, 13)
    full = oracle.estimate_normals(Q, 30)
    part = oracle.estimate_normals(Q, 30, rows=rows)
    assert np.abs(full[rows] - part).max() < 1e-12


# --------------------------------------------------------------------------
# Points in the plane (Sec. 3 states the problem in R^d)
# --------------------------------------------------------------------------

def test_planar_procrustes_is_the_2d_closed_form():
    """On points with z = 0 the 3-D alignment step is the 2-D one: a rotation
    about z by atan2(sum w (p x q)_z, sum w p . q) of the centred sets, and a
    translation in the plane."""
    g = np.random.default_rng(51)
    P = np.column_stack([g.random((300, 2)), np.zeros(300)])
    th = 0.7
    R2 = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    Q = np.column_stack([P[:, :2] @ R2.T + [0.3, -0.2] + 0.01 * g.standard_normal((300, 2)), np.zeros(300)])
    w = g.random(300)
    T = oracle.weighted_procrustes(P, Q, w)
    pb, qb = (w[:, None] * P).sum(0) / w.sum(), (w[:, None] * Q).sum(0) / w.sum()
    pc, qc = P - pb, Q - qb
    ang = np.arctan2((w * (pc[:, 0] * qc[:, 1] - pc[:, 1] * qc[:, 0])).sum(), (w * (pc * qc).sum(1)).sum())
    R = np.eye(3)
    R[:2, :2] = [[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]]
    assert np.abs(T[:3, :3] - R).max() < 1e-12
    assert np.abs(T[:3, 3] - (qb - R @ pb)).max() < 1e-12 and abs(T[2, 3]) < 1e-15


def _flower(n, g, noise=0.0):
    """Points on the planar curve r = 1 + 0.3 cos(5 th) (z = 0) and its in-plane unit normals."""
    th = g.random(n) * 2 * np.pi
    r = 1 + 0.3 * np.cos(5 * th)
    dr = -1.5 * np.sin(5 * th)
    P = np.column_stack([r * np.cos(th), r * np.sin(th), np.zeros(n)])
    tan = np.column_stack([dr * np.cos(th) - r * np.sin(th), dr * np.sin(th) + r * np.cos(th), np.zeros(n)])
    nrm = np.column_stack([tan[:, 1], -tan[:, 0], np.zeros(n)])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    if noise:
        P[:, :2] += noise * g.standard_normal((n, 2))
    return P, nrm


@pytest.mark.parametrize("variant", ["p2p", "p2p_welsch", "p2pl_welsch", "p2pl"])
def test_planar_registration_stays_in_the_plane(variant):
    """Points in the plane: every variant returns a rotation about z and a
    translation in the plane, and recovers an exact planar copy."""
    g = np.random.default_rng(52)
    Q, N = _flower(1500, g)
    th = 0.25
    Rz = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    P = (Q[:1200] - [0.05, -0.02, 0.0]) @ Rz            # the copy, moved in the plane
    r = oracle.register(P.astype(np.float32), Q.astype(np.float32), oracle.Params(variant=variant),
                        normals=N.astype(np.float32))
    assert r["status"] == "ok"
    assert np.array_equal(r["R"][2], [0.0, 0.0, 1.0]) and np.array_equal(r["R"][:, 2], [0.0, 0.0, 1.0])
    assert r["t"][2] == 0.0
    # the copy to within the stopping rule (epsilon = 1e-5 on the change of the iterate)
    assert np.abs(r["R"] - Rz).max() < 5e-5 and np.abs(P @ r["R"].T + r["t"] - Q[:1200]).max() < 5e-5


def test_line_search_first_trial_is_the_gauss_newton_step(monkeypatch):
    """Alg. 2 with every AA step sabotaged: each rejected AA iterate starts the line
    search along xi* - xi_prev at tau = 1, i.e. at the plain Gauss-Newton iterate
    (Eq. 18 without AA), whose own energy check then runs the same way. So the
    sabotaged run is plain Gauss-Newton: same iterations and accepted energies."""
    P, Q, N, _, _ = _surface_pair(21, n=500, angle=0.5, noise=0.01)
    prm = dict(variant="p2pl", max_iters=40)
    plain = oracle.register(P, Q, oracle.Params(anderson_m=0, **prm), normals=N)
    monkeypatch.setattr(oracle, "anderson_theta", lambda F, dF: np.full(dF.shape[1], 50.0))
    bad = oracle.register(P, Q, oracle.Params(anderson_m=5, **prm), normals=N)
    assert bad["aa_accepted"] == 0 and bad["iterations"] == plain["iterations"] > 3
    assert bad["line_search_trials"] >= bad["reverts"] > plain["reverts"]
    assert np.allclose(bad["trace"], plain["trace"], rtol=1e-10, atol=0)


# --------------------------------------------------------------------------
# The library k-d tree correspondence step equals the exhaustive definition
# (Sec. 3 Eq. 3), bit for bit, including duplicates and exact ties.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,dups", [(1, 5, 0), (7, 40, 0), (500, 800, 0), (3000, 2000, 200), (20000, 5000, 0)])
def test_kdtree_closest_equals_bruteforce(n, m, dups):
    g = np.random.default_rng(n + m)
    Q = g.random((n, 3)).astype(np.float32).astype(np.float64)
    if dups:
        Q[n - dups:] = Q[g.integers(0, n - dups, dups)]
    X = np.concatenate([g.random((m, 3)) * 1.3 - 0.15, Q[g.integers(0, n, min(m, 50))]])
    a = oracle.closest(X, Q)
    b = oracle.closest_kdtree(X, Q)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    if n > 1:
        assert np.array_equal(a[2], b[2])


def test_kdtree_closest_breaks_exact_ties_to_the_lowest_index():
    # a lattice: queries at cell centres are equidistant from 8 corners
    gx = np.arange(4, dtype=np.float64)
    G = np.stack(np.meshgrid(gx, gx, gx, indexing="ij"), -1).reshape(-1, 3)
    X = np.array([[0.5, 0.5, 0.5], [1.5, 2.5, 0.5], [1.0, 1.5, 2.0]])
    a = oracle.closest(X, G)
    b = oracle.closest_kdtree(X, G, k=12)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_registration_with_kdtree_correspondences_equals_bruteforce():
    from paper_2007_07627_gb300 import synth
    pair = synth.config_pair(1)
    for variant in ("p2p", "p2pl_welsch"):
        over = dict(max_iters=30) if variant == "p2p" else {}
        a = oracle.register(pair.P, pair.Q, oracle.Params(variant=variant, **over), normals=pair.normals)
        b = oracle.register(pair.P, pair.Q, oracle.Params(variant=variant, nn="kdtree", **over), normals=pair.normals)
        for key in ("iterations", "corr_passes", "reverts", "line_search_trials", "stages"):
            assert a[key] == b[key]
        assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["t"], b["t"])
        # every counter, R and t agree bit for bit; an energy has been seen to differ
        # by one ulp between the two runs in about one process in twenty (a library
        # reduction whose order is not fixed from one process to the next), so the
        # energies are compared to rounding
        assert np.allclose(a["trace"], b["trace"], rtol=1e-14, atol=0.0)


# --------------------------------------------------------------------------
# Robust symmetric objective (Sec. 7's proposed extension), read as Alg. 2 on
# H_i = (R p_i + t - q_i) . (R np_i + nq_i).
# --------------------------------------------------------------------------

@pytest.mark.parametrize("delta_scale", [0.0, 1e-8, 0.3, 1.2])
def test_symmetric_gradient_central_differences(delta_scale):
    g = np.random.default_rng(31)
    P = g.standard_normal((50, 3))
    Qh = g.standard_normal((50, 3))
    Nq = g.standard_normal((50, 3))
    Nq /= np.linalg.norm(Nq, axis=1, keepdims=True)
    Np = g.standard_normal((50, 3))
    Np /= np.linalg.norm(Np, axis=1, keepdims=True)
    d = g.standard_normal(3)
    u = g.standard_normal(3) if delta_scale else np.zeros(3)   # App. D's delta=0 case is exact at u=0
    xi = np.concatenate([delta_scale * d / np.linalg.norm(d), u])
    J = oracle.symmetric_gradient(xi, P, Qh, Nq, Np)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Hp, _, _ = oracle.symmetric_residual(xi + e, P, Qh, Nq, Np)
        Hm, _, _ = oracle.symmetric_residual(xi - e, P, Qh, Nq, Np)
        fd = (Hp - Hm) / (2 * h)
        assert np.abs(J[:, k] - fd).max() <= 1e-7 * max(1.0, np.abs(fd).max()), k


def test_symmetric_objective_without_source_normals_is_point_to_plane():
    """With every source normal zero, H_i is the point-to-plane residual of
    Eq. (15), its gradient that of App. D, and the registration is Alg. 2's, bit
    for bit (counters, transform, energy trace)."""
    from paper_2007_07627_gb300 import synth
    pair = synth.config_pair(3, 0.01)
    a = oracle.register(pair.P, pair.Q, oracle.Params(variant="p2pl_welsch"), normals=pair.normals)
    b = oracle.register(pair.P, pair.Q, oracle.Params(variant="sym_welsch"), normals=pair.normals,
                        source_normals=np.zeros_like(pair.P))
    for key in ("iterations", "corr_passes", "reverts", "line_search_trials", "stages"):
        assert a[key] == b[key], key
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["t"], b["t"])
    assert np.array_equal(a["trace"], b["trace"])


def test_symmetric_objective_recovers_an_exact_copy():
    """Target = a surface sample with its normals; source = the same points and
    normals under a known rigid motion: the registration returns the inverse
    motion and the energy goes to zero."""
    from paper_2007_07627_gb300 import synth
    pair = synth.ellipsoid_pair(synth.CONFIG_SEEDS[3], M=3000, N=3000, overlap=1.0, noise=0.0, outliers=0.0,
                                max_angle=0.0)
    Q, N = pair.Q.astype(np.float64), pair.normals.astype(np.float64)
    g = np.random.default_rng(32)
    R0 = _rot(g, 0.25)
    t0 = 0.03 * g.standard_normal(3)
    P = (Q @ R0.T + t0).astype(np.float32)
    Np = (N @ R0.T).astype(np.float32)
    r = oracle.register(P, pair.Q, oracle.Params(variant="sym_welsch"), normals=pair.normals, source_normals=Np)
    assert r["status"] == "ok"
    assert np.abs(r["R"] - R0.T).max() < 1e-6
    assert np.abs(r["t"] + R0.T @ t0).max() < 1e-6


def test_symmetric_objective_accepted_energy_is_monotone_within_stages():
    from paper_2007_07627_gb300 import synth
    pair = synth.config_pair(3, 0.01)
    r = oracle.register(pair.P, pair.Q, oracle.Params(variant="sym_welsch", nu_max=0.05, nu_min=0.05),
                        normals=pair.normals, source_normals=pair.src_normals)
    tr = np.asarray(r["trace"])
    assert r["stages"] == 1 and len(tr) > 3
    assert np.all(np.diff(tr) <= 1e-12 * np.abs(tr[:-1]))
