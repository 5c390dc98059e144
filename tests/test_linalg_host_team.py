"""The solver's small algebra run by teams of 7 and 32 host threads (one per
lane, a barrier as the team's sync) against a team of one lane, on the host:
the lane split and the exchange through the team scratch must give the same
bits for every routine, with every libm call the same on both sides (CPU only).
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

HERE = os.path.dirname(os.path.abspath(__file__))
IS, OS = 42, 36


@pytest.fixture(scope="module")
def T():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = os.path.join(HERE, "_build")   # in-tree, git-ignored
    os.makedirs(d, exist_ok=True)
    so = os.path.join(d, "liblinalg_host_team_threads.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-shared", "-x",
                    "cu", os.path.join(HERE, "linalg_host_team.cu"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.t_team_run.restype = ctypes.c_int
    L.t_team_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int]
    return L


def _run(L, op, lanes, cases):
    inp = np.zeros((len(cases), IS))
    for k, c in enumerate(cases):
        inp[k, :len(c)] = c
    out = np.zeros((len(cases), OS))
    assert L.t_team_run(op, lanes, len(cases), inp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), IS,
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), OS) == 0
    return out


def _cases(op, g):
    cases = []
    if op == 0:
        for k in range(60):
            mk = 1 + k % 5
            D = g.standard_normal((6, mk)) * 10.0 ** g.uniform(-6, 0)
            if k % 7 == 3:
                D[:, -1] = D[:, 0]
            cases.append(np.concatenate([[mk], D.ravel(), g.standard_normal(6)]))
    elif op == 1:
        for k in range(60):
            B = g.standard_normal((6, 6))
            A = B @ B.T + 10.0 ** g.uniform(-8, 0) * np.eye(6)
            b = g.standard_normal(6)
            if k % 4 == 1:
                z = g.choice(6, 3, replace=False)
                A[z, :] = 0.0
                A[:, z] = 0.0
                b[z] = 0.0
            if k % 9 == 2:
                A[5, 5] = -1.0
            cases.append(np.concatenate([A.ravel(), b]))
    elif op == 2:
        for k in range(40):
            P = g.standard_normal((30, 3))
            if k % 3 == 2:
                P[:, 2] = 0.0
            Q = P @ Rotation.random(random_state=k).as_matrix().T + 0.01 * g.standard_normal((30, 3))
            cases.append(((P - P.mean(0)).T @ (Q - Q.mean(0))).ravel())
    elif op in (3, 5):
        for s in (1.0, 0.3, 1e-3, 1e-5, 1e-7, 2.5, 0.0):
            for _ in range(6):
                cases.append(np.concatenate([g.standard_normal(3) * s, g.standard_normal(3)]))
    elif op == 4:
        for k in range(40):
            R = Rotation.random(random_state=100 + k).as_matrix()
            if k % 10 == 9:
                R = Rotation.from_rotvec(np.array([1.0, 2.0, 2.0]) / 3.0 * (np.pi - 1e-4)).as_matrix()
            cases.append(np.concatenate([R.ravel(), g.standard_normal(3)]))
    return cases


@pytest.mark.parametrize("op", [0, 1, 2, 3, 4, 5],
                         ids=["anderson", "chol6", "procrustes", "se3_exp", "se3_log", "p2pl_chain"])
def test_any_team_size_gives_the_bits_of_one_lane(T, op):
    cases = _cases(op, np.random.default_rng(80 + op))
    one = _run(T, op, 1, cases)
    for lanes in (7, 32):
        many = _run(T, op, lanes, cases)
        assert np.array_equal(many, one), (op, lanes, np.argwhere(many != one)[:5])
    assert np.isfinite(one).all()
