"""The oriented bucket boxes that prune the exact closest-point search (Eq. 3),
built for the host from the same source as the kernels (obb.cuh) and checked
against exact FP64 distances (CPU only). The search skips a bucket when the
box's float distance, shrunk by 2e-5, exceeds the running bound, so the box test
must never exceed (1 + 8e-6) times the squared distance to the bucket's nearest
point; and a bucket's own points must lie inside its box."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

HERE = os.path.dirname(os.path.abspath(__file__))
BOUND = 1.0 + 8e-6


@pytest.fixture(scope="module")
def H():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = os.path.join(HERE, "_build")   # in-tree, git-ignored
    os.makedirs(d, exist_ok=True)
    so = os.path.join(d, "libobb_host.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-x", "cu",
                    os.path.join(HERE, "obb_host.cu"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    fp = ctypes.POINTER(ctypes.c_float)
    L.h_obb_fit.argtypes = [fp, ctypes.c_int, fp]
    L.h_obb_d2.argtypes = [fp, fp, fp]
    L.h_obb_d2.restype = ctypes.c_float
    return L


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _fit(H, P32):
    pts = np.zeros((len(P32), 4), np.float32)
    pts[:, :3] = P32
    box = np.zeros(16, np.float32)
    H.h_obb_fit(_f(pts), len(P32), box.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return box


def _split(x):
    """x (FP64) as the search holds it: xh + xl, a float pair."""
    xh = x.astype(np.float32)
    xl = (x - xh.astype(np.float64)).astype(np.float32)
    return xh, xl


def _buckets(g):
    def patch(n, size, origin, curved=0.0, thick=0.0):
        uv = (g.random((n, 2)) - 0.5) * size
        z = curved * (uv ** 2).sum(1) + thick * g.standard_normal(n)
        P = np.column_stack([uv, z]) @ Rotation.random(random_state=g.integers(1 << 30)).as_matrix().T
        return (P + origin).astype(np.float32)

    base = g.random(3)
    yield "tilted plane", patch(16, 0.01, base)
    yield "curved patch", patch(16, 0.02, base, curved=3.0)
    yield "thick patch", patch(16, 0.01, base, thick=0.002)
    yield "blob", (base + 0.005 * g.standard_normal((16, 3))).astype(np.float32)
    yield "identical points", np.repeat(base[None].astype(np.float32), 16, 0)
    yield "collinear", (base + np.linspace(-0.01, 0.01, 16)[:, None] * g.standard_normal(3)).astype(np.float32)
    yield "one point", base[None].astype(np.float32)
    yield "two points", (base + 0.003 * g.standard_normal((2, 3))).astype(np.float32)
    yield "ragged 7", patch(7, 0.01, base, curved=1.0)
    yield "far from the origin", patch(16, 0.5, 1e4 * np.array([1.0, -0.3, 0.07]))
    yield "tiny patch off the origin", patch(16, 1e-3, 100.0 * np.ones(3))


@pytest.mark.parametrize("seed", range(6))
def test_bucket_points_lie_in_their_box(H, seed):
    g = np.random.default_rng(seed)
    zero = np.zeros(3, np.float32)
    for name, P in _buckets(g):
        box = _fit(H, P)
        for p in P:
            assert H.h_obb_d2(_f(box), _f(p), _f(zero)) == 0.0, name


@pytest.mark.parametrize("seed", range(6))
def test_box_distance_never_exceeds_the_nearest_point_distance(H, seed):
    g = np.random.default_rng(100 + seed)
    for name, P in _buckets(g):
        box = _fit(H, P)
        Pd = P.astype(np.float64)
        span = max(float(np.ptp(Pd, axis=0).max()), 1e-3)
        worst = 0.0
        for k in range(400):
            u = g.standard_normal(3)
            u /= np.linalg.norm(u)
            off = span * 10.0 ** g.uniform(-7, 2)             # from far inside float resolution to 100 spans
            x = Pd[g.integers(len(P))] + off * u
            xh, xl = _split(x)
            true = float((((xh.astype(np.float64) + xl) - Pd) ** 2).sum(1).min())
            got = float(H.h_obb_d2(_f(box), _f(xh), _f(xl)))
            assert got <= BOUND * true, (name, k, got, true)
            if true > 0.0:
                worst = max(worst, got / true)
            if off > 20 * span:                                # far: the box is no looser than the bucket
                assert got >= 0.5 * true, (name, got, true)
        assert worst <= BOUND
