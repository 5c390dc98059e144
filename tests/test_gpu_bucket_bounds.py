"""The oriented bucket boxes prune the exact closest-point search (Eq. 3)
without changing its result. Stress cases for the bound, each against the
oracle's brute force:

* targets on tilted planes (axis-aligned boxes are loose there, oriented ones
  tight) with queries at normal offsets from 1e-7 to 0.3 of the plane size,
  exact copies of target points and far queries;
* the same geometry far from the origin (coordinates ~1e4), where the float
  rounding of the box test is largest next to the bucket size;
* degenerate buckets: many copies of one point, collinear runs;
* the per-thread search (fricp_closest_points), the warp search (one pass
  through fricp_eval_pass) and query tiles (every pass of a registration,
  through its step records).
"""
import numpy as np
import pytest

import oracle
from tests.gpu_common import assert_nn_parity, oracle_pass_p2p

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2007_07627_gb300 import build
    build.build()
    import paper_2007_07627_gb300 as fr
    fr.lib()
    return fr


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _planes(g, n_planes=6, per=4000, size=0.6):
    """Points on tilted square patches; returns points and the patch normals."""
    pts, nrm = [], []
    for _ in range(n_planes):
        n = _unit(g.standard_normal(3))
        e1 = _unit(np.cross(n, g.standard_normal(3)))
        e2 = np.cross(n, e1)
        uv = (g.random((per, 2)) - 0.5) * size
        pts.append(g.random(3) + uv[:, :1] * e1 + uv[:, 1:] * e2)
        nrm.append(np.repeat(n[None], per, 0))
    return np.concatenate(pts), np.concatenate(nrm)


def _queries(g, Q, nQ, size=0.6):
    """Target points moved along their normal by 1e-7 .. 0.3 x size, exact copies,
    and far points."""
    k = len(Q)
    sel = g.choice(k, 3000, replace=False)
    off = size * 10.0 ** g.uniform(-7, np.log10(0.3), 3000)
    sgn = np.where(g.random(3000) < 0.5, -1.0, 1.0)
    near = Q[sel] + (sgn * off)[:, None] * nQ[sel]
    copies = Q[g.choice(k, 300, replace=False)]
    lo, hi = Q.min(0), Q.max(0)
    far = lo - 0.5 + (hi - lo + 1.0) * g.random((700, 3))
    return np.concatenate([near, copies, far])


def _check_closest(fr, Q32, P32, T=None):
    t = fr.target_create(Q32)
    idx, d2 = fr.closest_points(t, _dev(P32), T)
    X = P32.astype(float) if T is None else oracle.apply(T, P32.astype(float))
    io, do, dso = oracle.closest(X, Q32.astype(float))
    return assert_nn_parity(idx.cpu().numpy(), d2.cpu().numpy(), io, do, dso)


@pytest.mark.parametrize("origin", [0.0, 1e4])
def test_closest_points_tilted_planes(fr, origin):
    g = np.random.default_rng(11)
    Q, nQ = _planes(g)
    P = _queries(g, Q, nQ)
    scale = 50.0 if origin else 1.0       # coordinates ~1e4: patches 30 wide, points ~0.5 apart
    shift = origin * np.array([1.0, -0.3, 0.07])
    Q32 = (Q * scale + shift).astype(np.float32)
    P32 = (P * scale + shift).astype(np.float32)
    _check_closest(fr, Q32, P32)


def test_closest_points_degenerate_buckets(fr):
    g = np.random.default_rng(12)
    line = np.linspace(0.0, 1.0, 200)[:, None] * np.array([0.3, -0.2, 0.5]) + 0.1
    same = np.repeat(np.array([[0.7, 0.2, 0.4]]), 40, 0)
    flat = np.column_stack([g.random(500), g.random(500), np.full(500, 0.25)])
    Q = np.concatenate([line, same, flat, g.random((300, 3))])
    P = np.concatenate([Q[g.choice(len(Q), 400)] + 1e-5 * g.standard_normal((400, 3)),
                        g.random((600, 3)) * 1.4 - 0.2, same[:3]])
    _check_closest(fr, Q.astype(np.float32), P.astype(np.float32))


def test_warp_search_pass_on_tilted_planes(fr):
    """One fused point-to-point pass (the warp search) on the tilted planes:
    the energy is the oracle's to 1e-10, so every correspondence is."""
    g = np.random.default_rng(13)
    Q, nQ = _planes(g, per=3000)
    P = _queries(g, Q, nQ)
    Q32, P32 = Q.astype(np.float32), P.astype(np.float32)
    t = fr.target_create(Q32)
    nz = oracle.normalization(P32.astype(float), Q32.astype(float))
    for Tn in (np.eye(4), np.array([[1, 0, 0, 0.01], [0, 1, 0, -0.02], [0, 0, 1, 0.005], [0, 0, 0, 1.0]])):
        out = fr.eval_pass(t, P32, "p2p", Tn, scale=nz.s, center=nz.c)
        E_o, _ = oracle_pass_p2p(P32, Q32, Tn, 1.0, nz.s, nz.c, robust=False)
        assert abs(out[0] - E_o) <= 1e-10 * E_o, (out[0], E_o)


def test_query_tiles_every_pass_on_tilted_planes(fr):
    """Point-to-point registration searched by query tiles: every recorded
    pass's energy equals the oracle's pass at the recorded transform."""
    g = np.random.default_rng(14)
    Q, nQ = _planes(g, per=3000)
    P = _queries(g, Q, nQ)
    Q32, P32 = Q.astype(np.float32), P.astype(np.float32)
    t = fr.target_create(Q32)
    prm = fr.params_default("p2p", search=0, max_iters=15)     # FRICP_SEARCH_TILE
    res, steps = fr.register_recorded(t, P32, params=prm, steps_capacity=256)
    assert res["status"] == "OK" and len(steps) > 3
    nz = oracle.normalization(P32.astype(float), Q32.astype(float))
    for s in steps:
        E_o, _ = oracle_pass_p2p(P32, Q32, s["T"], 1.0, nz.s, nz.c, robust=False)
        assert abs(s["E"] - E_o) <= 1e-10 * E_o, (s["step"], s["E"], E_o)
