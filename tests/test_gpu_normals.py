"""GPU normal estimate (fricp_estimate_normals) against the FP64 oracle's
reading of Sec. 6 (PCA over the k nearest neighbours, the point included).

Normals are unique where the neighbourhood's two smallest covariance
eigenvalues are apart; there the GPU normal (stored as float32) must match the
oracle's to 1e-6 and its orientation too, unless the point sees the viewpoint
edge-on. Where the eigenvalues nearly coincide any vector of that eigenspace
is correct, so only its Rayleigh quotient is checked.
"""
import numpy as np
import pytest

import oracle
from paper_2007_07627_gb300 import synth
from tests.gpu_common import assert_registration_parity, oracle_reference

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


def _assert_normals(Q, got, k, viewpoint=None, rows=None):
    Q64 = Q.astype(np.float64)
    rows = np.arange(Q.shape[0]) if rows is None else np.asarray(rows)
    ref = oracle.estimate_normals(Q64, k, viewpoint, rows=rows)
    g = got[rows].astype(np.float64)
    assert np.abs(np.linalg.norm(g, axis=1) - 1.0).max() < 1e-6
    idx, _ = oracle.knn_query(Q64[rows], Q64, k)
    nb = Q64[idx]
    c = nb.mean(axis=1, keepdims=True)
    C = np.einsum("nki,nkj->nij", nb - c, nb - c) / nb.shape[1]
    ev = np.linalg.eigvalsh(C)
    unique = (ev[:, 1] - ev[:, 0]) > 1e-6 * np.maximum(ev[:, 2], 1e-300)
    v = np.zeros(3) if viewpoint is None else np.asarray(viewpoint, np.float64)
    to_v = v[None, :] - Q64[rows]
    edge_on = np.abs(np.einsum("nd,nd->n", ref, to_v)) < 1e-6 * np.linalg.norm(to_v, axis=1)
    dots = np.einsum("nd,nd->n", g, ref)
    strict = unique & ~edge_on
    assert (dots[strict] > 1.0 - 1e-6).all(), np.sort(dots[strict])[:5]
    assert (np.abs(dots[unique]) > 1.0 - 1e-6).all()
    rq = np.einsum("nd,nde,ne->n", g, C, g)
    assert (rq[~unique] <= ev[~unique, 0] + 1e-6 * np.maximum(ev[~unique, 2], 1e-300)).all()
    return int(unique.sum())


@pytest.mark.parametrize("n,k", [(5, 30), (17, 6), (31, 30), (33, 32), (500, 3), (2000, 30)])
def test_normals_small_and_ragged(fr, n, k):
    g = np.random.default_rng(n + k)
    Q = (g.random((n, 3)) * [1.0, 0.8, 0.1]).astype(np.float32)
    _assert_normals(Q, fr.estimate_normals(Q, k), min(k, n))


def test_normals_of_a_tilted_plane(fr):
    g = np.random.default_rng(41)
    xy = g.random((4000, 2))
    Q = np.column_stack([xy, 0.3 * xy[:, 0] - 0.7 * xy[:, 1] + 0.2]).astype(np.float32)
    v = [0.5, 0.5, 5.0]
    N = fr.estimate_normals(Q, 30, viewpoint=v)
    _assert_normals(Q, N, 30, v)
    n_true = np.array([-0.3, 0.7, 1.0]) / np.linalg.norm([-0.3, 0.7, 1.0])
    assert (N.astype(np.float64) @ n_true > 1 - 1e-5).all()


def test_normals_with_duplicate_points(fr):
    g = np.random.default_rng(42)
    Q = g.random((800, 3)).astype(np.float32)
    Q[700:760] = Q[g.integers(0, 700, 60)]
    _assert_normals(Q, fr.estimate_normals(Q, 30), 30)


@pytest.mark.parametrize("cfg,scale", [(2, 0.05), (3, 0.02)])
def test_normals_of_workload_targets(fr, cfg, scale):
    pair = synth.config_pair(cfg, scale)
    N = fr.estimate_normals(pair.Q, 30)
    assert _assert_normals(pair.Q, N, 30) > 0.9 * pair.N
    # the analytic normals of the generator agree up to sign and the surface's curvature
    cos = np.abs(np.einsum("nd,nd->n", N.astype(np.float64), pair.normals.astype(np.float64)))
    assert np.median(cos) > 0.99


def test_normals_device_and_host_agree(fr):
    import torch
    pair = synth.config_pair(3, 0.01)
    a = fr.estimate_normals(pair.Q, 30)
    b = fr.estimate_normals(torch.from_numpy(pair.Q).cuda(), 30).cpu().numpy()
    assert np.array_equal(a, b)


def test_normals_of_full_size_workload3_target_sampled(fr):
    """All 500,000 points of workload 3's target on the GPU; 2,000 sampled
    points checked against the oracle's neighbourhoods over the whole set."""
    pair = synth.config_pair(3)
    N = fr.estimate_normals(pair.Q, 30)
    rows = np.random.default_rng(43).choice(pair.N, 2000, replace=False)
    _assert_normals(pair.Q, N, 30, rows=rows)


def test_point_to_plane_with_estimated_normals(fr):
    """Alg. 2 on estimated normals: GPU normals + GPU registration against oracle
    normals + oracle registration (the normals match to float rounding)."""
    pair = synth.ellipsoid_pair(synth.CONFIG_SEEDS[3], M=3000, N=8000, overlap=1.0, outliers=0.0)
    Ng = fr.estimate_normals(pair.Q, 30)
    No = oracle.estimate_normals(pair.Q.astype(np.float64), 30).astype(np.float32)
    assert np.abs(np.abs(np.einsum("nd,nd->n", Ng, No)) - 1.0).max() < 1e-5
    t = fr.target_create(pair.Q, Ng)
    r = fr.register(t, pair.P, params=fr.params_default("p2pl_welsch"), trace_capacity=4096)
    est = synth.Pair(P=pair.P, Q=pair.Q, normals=Ng, R_gt=pair.R_gt, t_gt=pair.t_gt, diag=pair.diag)
    ref = oracle_reference(est, "p2pl_welsch", {}, perms=(1, 2))
    assert_registration_parity(r, ref, pair.diag)
    t.destroy()


def test_normal_estimate_argument_errors(fr):
    Q = np.zeros((10, 3), np.float32)
    for k in (2, 33):
        with pytest.raises(fr.FricpError):
            fr.estimate_normals(Q, k)
    Q[3, 1] = np.nan
    with pytest.raises(fr.FricpError):
        fr.estimate_normals(Q, 6)
