"""Points in the plane (Sec. 3 states the problem in R^d) registered as 3-D
points with z = 0, on the GPU against the oracle: every variant returns a
rotation about z and a translation in the plane, and matches the oracle."""
import numpy as np
import pytest

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


def _flower_pair(seed, n_q=3000, n_p=2400, noise=0.004, outliers=0.0, angle=0.3):
    g = np.random.default_rng(seed)

    def curve(n):
        th = g.random(n) * 2 * np.pi
        r = 1 + 0.3 * np.cos(5 * th)
        dr = -1.5 * np.sin(5 * th)
        P = np.column_stack([r * np.cos(th), r * np.sin(th), np.zeros(n)])
        tan = np.column_stack([dr * np.cos(th) - r * np.sin(th), dr * np.sin(th) + r * np.cos(th), np.zeros(n)])
        nrm = np.column_stack([tan[:, 1], -tan[:, 0], np.zeros(n)])
        return P, nrm / np.linalg.norm(nrm, axis=1, keepdims=True)

    Q, N = curve(n_q)
    S, _ = curve(n_p)
    S[:, :2] += noise * g.standard_normal((n_p, 2))
    k = int(outliers * n_p)
    if k:
        S[:k, :2] = g.uniform(-1.4, 1.4, (k, 2))
    Rz = np.array([[np.cos(angle), -np.sin(angle), 0], [np.sin(angle), np.cos(angle), 0], [0, 0, 1.0]])
    t = np.array([0.05, -0.03, 0.0])
    P = S @ Rz.T + t
    return synth.Pair(P=P.astype(np.float32), Q=Q.astype(np.float32), normals=N.astype(np.float32),
                      R_gt=Rz.T.copy(), t_gt=-(Rz.T @ t), diag=float(np.linalg.norm(Q.max(0) - Q.min(0))),
                      name="flower")


@pytest.mark.parametrize("variant,outliers", [("p2p", 0.0), ("p2p_welsch", 0.1), ("p2pl_welsch", 0.1),
                                              ("p2pl", 0.0)])
def test_planar_registration_matches_oracle(fr, variant, outliers):
    pair = _flower_pair(61, outliers=outliers)
    over = {"max_iters": 200} if variant in ("p2p", "p2pl") else {}
    t = fr.target_create(pair.Q, pair.normals if variant.startswith("p2pl") else None)
    r = fr.register(t, pair.P, params=fr.params_default(variant, **over), trace_capacity=20000)
    assert np.array_equal(r["R"][2], [0.0, 0.0, 1.0]) and np.array_equal(r["R"][:, 2], [0.0, 0.0, 1.0])
    assert r["t"][2] == 0.0
    ref = oracle_reference(pair, variant, over, perms=(1, 2, 3, 4), jitters=2)
    assert_registration_parity(r, ref, pair.diag)
    t.destroy()
