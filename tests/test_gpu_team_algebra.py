"""The solver's small algebra run by a team of 32 lanes on the GPU against the
same routines run serially on the host (a team of one lane): the lane split
and the shared-scratch exchange must not change a bit of the arithmetic.

Anderson least squares and the 6x6 Cholesky solve use only +, *, fma and the
float-seeded reciprocals, so device and host agree bit for bit. The routines
with sin/cos/atan2 (Procrustes polish, SE(3) exp/log, the App. D chain
matrix) agree to the math libraries' last-bit differences.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
IS, OS = 42, 36


@pytest.fixture(scope="module")
def libs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = os.path.join(HERE, "_build")   # in-tree, git-ignored
    os.makedirs(d, exist_ok=True)
    host = os.path.join(d, "liblinalg_host_team.so")   # its own file: another test may hold liblinalg_host.so
    dev = os.path.join(d, "liblinalg_device.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-x", "cu",
                    os.path.join(HERE, "linalg_host.cu"), "-o", host], check=True)
    subprocess.run([nvcc, "-O3", "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                    "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC", "-shared",
                    os.path.join(HERE, "linalg_device.cu"), "-o", dev], check=True)
    H, D = ctypes.CDLL(host), ctypes.CDLL(dev)
    dp = ctypes.POINTER(ctypes.c_double)
    for n in ("h_procrustes_rotation", "h_anderson_lstsq", "h_chol6_solve"):
        getattr(H, n).restype = ctypes.c_int
    H.h_procrustes_rotation.argtypes = [dp, dp]
    H.h_se3_exp.argtypes = [dp, dp]
    H.h_se3_log.argtypes = [dp, dp]
    H.h_anderson_lstsq.argtypes = [dp, dp, ctypes.c_int, dp]
    H.h_chol6_solve.argtypes = [dp, dp, dp]
    H.h_p2pl_chain.argtypes = [dp, dp]
    D.d_team_run.restype = ctypes.c_int
    D.d_team_run.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int]
    return H, D


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _device(D, op, cases):
    inp = np.zeros((len(cases), IS))
    for k, c in enumerate(cases):
        inp[k, :len(c)] = c
    out = np.zeros((len(cases), OS))
    assert D.d_team_run(op, len(cases), _p(inp), IS, _p(out), OS) == 0
    return out


def test_anderson_lstsq_bit_identical(libs):
    H, D = libs
    g = np.random.default_rng(71)
    cases, host = [], []
    for k in range(200):
        mk = 1 + k % 5
        Dm = g.standard_normal((6, mk)) * 10.0 ** g.uniform(-6, 0)
        if k % 7 == 3:
            Dm[:, -1] = Dm[:, 0] * (1 + 1e-15)          # rank rule
        if k % 11 == 5:
            Dm[:3] *= 1e-9                             # badly scaled rows
        f = g.standard_normal(6)
        th = np.zeros(5)
        ok = H.h_anderson_lstsq(_p(np.ascontiguousarray(Dm)), _p(f), mk, _p(th))
        cases.append(np.concatenate([[mk], Dm.ravel(), f]))
        host.append(np.concatenate([[ok], th[:mk]]))
    dev = _device(D, 0, cases)
    for k, h in enumerate(host):
        n = len(h) if h[0] == 1.0 else 1      # theta is only defined when the solve succeeds
        assert np.array_equal(dev[k, :n], h[:n]), (k, dev[k, :n], h[:n])
    assert 0 < sum(h[0] for h in host) < len(host)


def test_chol6_bit_identical_including_zero_directions(libs):
    H, D = libs
    g = np.random.default_rng(72)
    cases, host = [], []
    for k in range(200):
        B = g.standard_normal((6, 6))
        A = B @ B.T + 10.0 ** g.uniform(-8, 0) * np.eye(6)
        b = g.standard_normal(6)
        if k % 4 == 1:                                 # planar system: three exactly-zero directions
            z = g.choice(6, 3, replace=False)
            A[z, :] = 0.0
            A[:, z] = 0.0
            b[z] = 0.0
        if k % 9 == 2:
            A[5, 5] = -1.0                             # not positive definite
        x = np.zeros(6)
        ok = H.h_chol6_solve(_p(np.ascontiguousarray(A)), _p(b), _p(x))
        cases.append(np.concatenate([A.ravel(), b]))
        host.append(np.concatenate([[ok], x]))
    dev = _device(D, 1, cases)
    for k, h in enumerate(host):
        n = 7 if h[0] == 1.0 else 1           # x is only defined when the solve succeeds
        assert np.array_equal(dev[k, :n], h[:n]), (k, dev[k, :n], h[:n])
    assert 0 < sum(h[0] for h in host) < len(host)


def _close(a, b, tol):
    return np.abs(a - b).max() <= tol * max(1.0, np.abs(b).max())


def test_transcendental_routines_agree(libs):
    H, D = libs
    g = np.random.default_rng(73)
    from scipy.spatial.transform import Rotation
    # Procrustes
    cases, host = [], []
    for k in range(100):
        P = g.standard_normal((30, 3))
        if k % 3 == 2:
            P[:, 2] = 0.0
        Q = P @ Rotation.random(random_state=k).as_matrix().T + 0.01 * g.standard_normal((30, 3))
        Hm = (P - P.mean(0)).T @ (Q - Q.mean(0))
        R = np.zeros(9)
        ok = H.h_procrustes_rotation(_p(np.ascontiguousarray(Hm)), _p(R))
        cases.append(Hm.ravel())
        host.append(np.concatenate([[ok], R]))
    dev = _device(D, 2, cases)
    for k, h in enumerate(host):
        assert dev[k, 0] == h[0] and _close(dev[k, 1:10], h[1:], 2e-15), k
    # exp, log, chain
    xis = [np.concatenate([g.standard_normal(3) * s, g.standard_normal(3)]) for s in
           (1.0, 0.3, 1e-3, 1e-5, 1e-7, 2.5) for _ in range(10)]
    dev_T = _device(D, 3, xis)
    dev_K = _device(D, 5, xis)
    for k, xi in enumerate(xis):
        T, K = np.zeros(12), np.zeros(36)
        H.h_se3_exp(_p(np.ascontiguousarray(xi)), _p(T))
        H.h_p2pl_chain(_p(np.ascontiguousarray(xi)), _p(K))
        assert _close(dev_T[k, :12], T, 2e-15), k
        assert _close(dev_K[k, :36], K, 1e-14), k
    dev_xi = _device(D, 4, [dev_T[k, :12] for k in range(len(xis))])
    for k in range(len(xis)):
        back = np.zeros(6)
        H.h_se3_log(_p(np.ascontiguousarray(dev_T[k, :12])), _p(back))
        assert _close(dev_xi[k, :6], back, 1e-14), k
