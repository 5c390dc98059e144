"""The CUDA path's small FP64 algebra (procrustes rotation, exp/log on SE(3),
Anderson least squares, 6x6 Cholesky, App. D chain matrix) compiled for the host
and compared with numpy / scipy and the oracle (CPU only)."""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.spatial.transform import Rotation

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def H():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = os.path.join(HERE, "_build")   # in-tree, git-ignored
    os.makedirs(d, exist_ok=True)
    so = os.path.join(d, "liblinalg_host.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-x", "cu",
                    os.path.join(HERE, "linalg_host.cu"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    for n in ("h_procrustes_rotation", "h_anderson_lstsq", "h_chol6_solve"):
        getattr(L, n).restype = ctypes.c_int
    L.h_procrustes_rotation.argtypes = [dp, dp]
    L.h_se3_exp.argtypes = [dp, dp]
    L.h_se3_log.argtypes = [dp, dp]
    L.h_anderson_lstsq.argtypes = [dp, dp, ctypes.c_int, dp]
    L.h_chol6_solve.argtypes = [dp, dp, dp]
    L.h_p2pl_chain.argtypes = [dp, dp]
    return L


def _p(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _T12(T):
    return np.concatenate([T[:3, :3].ravel(), T[:3, 3]])


def test_procrustes_rotation_matches_svd_kabsch(H):
    g = np.random.default_rng(1)
    for trial in range(300):
        P = g.standard_normal((40, 3))
        if trial % 3 == 1:
            P[:, 2] *= 1e-3                      # nearly planar
        if trial % 3 == 2:
            P[:, 2] = 0.0                        # exactly planar: rank 2
        R0 = Rotation.random(random_state=trial).as_matrix()
        Q = P @ R0.T + 0.01 * g.standard_normal((40, 3))
        w = g.random(40)
        T = oracle.weighted_procrustes(P, Q, w)
        pb = (w[:, None] * P).sum(0) / w.sum()
        qb = (w[:, None] * Q).sum(0) / w.sum()
        Hm = np.ascontiguousarray(((P - pb) * w[:, None]).T @ (Q - qb))
        R = np.zeros(9)
        assert H.h_procrustes_rotation(_p(Hm), _p(R)) == 1
        R = R.reshape(3, 3)
        assert np.abs(R - T[:3, :3]).max() < 1e-12, trial
        assert abs(np.linalg.det(R) - 1) < 1e-13


def test_procrustes_rotation_rejects_rank_one(H):
    Hm = np.outer([1.0, 2.0, 3.0], [0.5, -1.0, 2.0])
    R = np.zeros(9)
    assert H.h_procrustes_rotation(_p(Hm), _p(R)) == 0


@pytest.mark.parametrize("scale", [3.0, 1.0, 0.1, 1e-3, 1e-6, 1e-9, 0.0])
def test_se3_exp_log_match_scipy(H, scale):
    g = np.random.default_rng(2)
    for _ in range(100):
        a = g.standard_normal(3)
        a = a / np.linalg.norm(a) * scale * (0.5 + 0.5 * g.random()) if scale else np.zeros(3)
        xi = np.concatenate([a, g.standard_normal(3)])
        T = np.zeros(12)
        H.h_se3_exp(_p(xi), _p(T))
        Tref = oracle.se3_exp(oracle.se3_matrix(xi))
        assert np.abs(T - _T12(Tref)).max() < 1e-14
        back = np.zeros(6)
        H.h_se3_log(_p(_T12(Tref)), _p(back))
        assert np.abs(back - xi).max() < 1e-12, (scale, back - xi)


def test_se3_log_near_pi(H):
    for ang in (math.pi - 1e-4, math.pi - 1e-8):
        a = np.array([0.3, -0.4, 0.5])
        xi = np.concatenate([a / np.linalg.norm(a) * ang, [0.1, 0.2, 0.3]])
        Tref = oracle.se3_exp(oracle.se3_matrix(xi))
        back = np.zeros(6)
        H.h_se3_log(_p(_T12(Tref)), _p(back))
        T2 = oracle.se3_exp(oracle.se3_matrix(back))
        assert np.abs(T2 - Tref).max() < 1e-7


def test_anderson_lstsq_matches_numpy(H):
    g = np.random.default_rng(3)
    for mk in range(1, 6):
        D = g.standard_normal((6, mk))
        f = g.standard_normal(6)
        th = np.zeros(5)
        assert H.h_anderson_lstsq(_p(D), _p(f), mk, _p(th)) == 1
        ref = np.linalg.lstsq(D, f, rcond=None)[0]
        assert np.abs(th[:mk] - ref).max() < 1e-12
    D = np.ones((6, 2))
    assert H.h_anderson_lstsq(_p(D), _p(np.ones(6)), 2, _p(np.zeros(5))) == 0


def test_chol6_matches_numpy(H):
    g = np.random.default_rng(4)
    A = g.standard_normal((6, 6))
    A = A @ A.T + 0.1 * np.eye(6)
    b = g.standard_normal(6)
    x = np.zeros(6)
    assert H.h_chol6_solve(_p(A), _p(b), _p(x)) == 1
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-12
    A[5, 5] = -1.0
    assert H.h_chol6_solve(_p(A), _p(b), _p(x)) == 0


def test_chol6_zero_directions_are_the_reduced_system(H):
    """Points in a plane: the directions with an all-zero row, column and
    right-hand side get x_j = 0 and the rest solves the reduced system."""
    g = np.random.default_rng(6)
    keep = np.array([2, 3, 4])
    B = g.standard_normal((3, 3))
    A = np.zeros((6, 6))
    A[np.ix_(keep, keep)] = B @ B.T + 0.1 * np.eye(3)
    b = np.zeros(6)
    b[keep] = g.standard_normal(3)
    x = np.full(6, np.nan)
    assert H.h_chol6_solve(_p(A), _p(b), _p(x)) == 1
    ref = np.zeros(6)
    ref[keep] = np.linalg.solve(A[np.ix_(keep, keep)], b[keep])
    assert np.abs(x - ref).max() < 1e-12 and (x[[0, 1, 5]] == 0.0).all()
    assert H.h_chol6_solve(_p(np.zeros((6, 6))), _p(np.zeros(6)), _p(x)) == 0
    b[0] = 1.0                                   # a zero row with a nonzero right-hand side is singular
    assert H.h_chol6_solve(_p(A), _p(b), _p(x)) == 0


def test_procrustes_rotation_rejects_non_finite(H):
    Hm = np.eye(3)
    R = np.zeros(9)
    for bad in (np.nan, np.inf):
        Hm[1, 2] = bad
        assert H.h_procrustes_rotation(_p(Hm), _p(R)) == 0


@pytest.mark.parametrize("scale", [1.0, 0.2, 1e-4, 1e-8, 0.0])
def test_chain_matrix_reproduces_appendix_d_gradient(H, scale):
    """J_i = K z_i with z_i = [R p_i x n_i; n_i] equals the oracle's App. D gradient."""
    g = np.random.default_rng(5)
    d = g.standard_normal(3)
    d = d / np.linalg.norm(d) * scale if scale else np.zeros(3)
    u = g.standard_normal(3) if scale else np.zeros(3)
    xi = np.concatenate([d, u])
    P = g.standard_normal((20, 3))
    N = g.standard_normal((20, 3))
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    K = np.zeros(36)
    H.h_p2pl_chain(_p(xi), _p(K))
    K = K.reshape(6, 6)
    R = sla.expm(oracle.hat(d))
    y = P @ R.T
    z = np.concatenate([np.cross(y, N), N], axis=1)
    J = z @ K.T
    Jref = oracle.plane_gradient(xi, P, N)
    assert np.abs(J - Jref).max() < 1e-9 * max(1.0, np.abs(Jref).max())
