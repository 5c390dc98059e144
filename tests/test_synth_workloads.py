"""The seeded synthetic workloads against the recipe they stand for (CPU only):
the surfaces, sizes, noise, outlier and overlap shares, motion bounds and the
source normals of workloads 1-3, and the ranges of the batched and served mixes.
The paper's scans are not available, so these pairs stand in for them; this
pins that they have the stated shape."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2007_07627_gb300 import synth


def _angle_deg(R):
    return math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1.0) / 2.0))))


def _aligned(pair):
    """The source moved back onto the target by the ground-truth motion."""
    return pair.P.astype(np.float64) @ pair.R_gt.T + pair.t_gt


def test_workload1_torus():
    pair = synth.config_pair(1)
    assert (pair.N, pair.M) == (2000, 2000)
    Q = pair.Q.astype(np.float64)
    ring = np.hypot(Q[:, 0], Q[:, 1]) - 1.0                  # torus R = 1, r = 0.4
    assert np.abs(np.hypot(ring, Q[:, 2]) - 0.4).max() < 1e-6
    X = _aligned(pair)
    ring = np.hypot(X[:, 0], X[:, 1]) - 1.0
    resid = np.hypot(ring, X[:, 2]) - 0.4                    # full overlap, no outliers: noise only
    assert resid.std() == pytest.approx(0.002 * pair.diag, rel=0.1)
    assert _angle_deg(pair.R_gt) <= 30.0 + 1e-9
    assert np.linalg.norm(pair.t_gt) <= 0.1 * pair.diag * math.sqrt(3) + 1e-9   # translation within 0.1 diag per axis


@pytest.mark.parametrize("cfg,N,M,noise,outliers,overlap,max_angle", [
    (2, 100_000, 80_000, 0.005, 0.10, 0.6, 25.0),
    (3, 500_000, 200_000, 0.003, 0.05, 0.5, 25.0)])
def test_workloads_2_3_shape(cfg, N, M, noise, outliers, overlap, max_angle):
    scale = 0.05
    pair = synth.config_pair(cfg, scale)
    assert (pair.N, pair.M) == (int(N * scale), int(M * scale))
    full = synth.config_pair(cfg, 1.0) if cfg == 2 else None
    if full is not None:
        assert (full.N, full.M) == (N, M)
    assert _angle_deg(pair.R_gt) <= max_angle + 1e-9
    X = _aligned(pair)
    d, _ = cKDTree(pair.Q.astype(np.float64)).query(X)
    near = d < 4.0 * noise * pair.diag
    # surface points inside the overlap sit within the noise of the target; the
    # rest (the cropped share and the outliers) lie farther out
    share_near = float(near.mean())
    assert share_near == pytest.approx(overlap * (1.0 - outliers), abs=0.12)
    # noise: the normal offset of the near points (the target is dense enough that
    # the nearest target point is about the foot of the normal)
    if pair.normals is not None and cfg == 3:
        _, j = cKDTree(pair.Q.astype(np.float64)).query(X[near])
        h = np.einsum("nd,nd->n", X[near] - pair.Q[j].astype(np.float64), pair.normals[j].astype(np.float64))
        assert h.std() == pytest.approx(noise * pair.diag, rel=0.25)


def test_workload3_normals_and_source_normals():
    pair = synth.config_pair(3, 0.02)
    n = pair.normals.astype(np.float64)
    assert np.abs(np.linalg.norm(n, axis=1) - 1.0).max() < 1e-5
    ns = pair.src_normals.astype(np.float64)
    assert np.abs(np.linalg.norm(ns, axis=1) - 1.0).max() < 1e-5
    # a source normal moved back by the ground truth matches the target normal at
    # its surface point (inside the overlap, away from the outliers)
    X = _aligned(pair)
    d, j = cKDTree(pair.Q.astype(np.float64)).query(X)
    near = d < 2.0 * 0.003 * pair.diag
    back = ns[near] @ pair.R_gt.T
    cosang = np.einsum("nd,nd->n", back, n[j[near]])
    assert np.median(cosang) > 0.99


def test_batched_and_served_mixes():
    specs = synth.batch_specs()
    assert len(specs) == 256
    Ms = np.array([s["M"] for s in specs])
    Ns = np.array([s["N"] for s in specs])
    assert Ms.min() >= 2000 and Ms.max() <= 200_000 and Ns.min() >= 2000 and Ns.max() <= 200_000
    # log-uniform: the median is near the geometric mean of the range
    assert np.median(np.log(Ms)) == pytest.approx(math.log(math.sqrt(2000 * 200_000)), abs=0.5)
    variants = [s["variant"] for s in specs]
    assert sorted(set(variants)) == sorted(synth.BATCH_VARIANTS)
    assert max(variants.count(v) for v in set(variants)) - min(variants.count(v) for v in set(variants)) <= 1
    assert {s["kind"] for s in specs} == {0, 1, 2}
    assert all(0.5 <= s["overlap"] <= 1.0 and 0.0 <= s["outliers"] <= 0.1 for s in specs)
    serve = synth.serve_specs(n=64)
    assert all(1000 <= s["M"] <= 1_000_000 and 1000 <= s["N"] <= 1_000_000 for s in serve)
    assert {s["variant"] for s in serve} == set(synth.SERVE_VARIANTS)
