"""The two layouts of the exact closest-point search (Eq. 3) give the same
argmin, so whole registrations are identical bit for bit: query tiles (a warp
per 32 Morton-adjacent queries, buckets staged in shared memory, the default)
against one query per warp. Covers every variant and precision mode, ragged
tile tails, sources far from the target (tiles whose candidate list does not
fit and fall back to per-query search), the full-size workloads 2 and 3, and
the batched engine."""
import numpy as np
import pytest

from paper_2007_07627_gb300 import synth

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


def _same(a, b):
    assert a["status"] == b["status"]
    for key in ("iterations", "corr_passes", "aa_accepted", "reverts", "line_search_trials", "stages",
                "device_steps"):
        assert a[key] == b[key], (key, a[key], b[key])
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["t"], b["t"])
    assert a["final_energy"] == b["final_energy"]
    assert np.array_equal(a["trace"], b["trace"])


def _both(fr, t, P, variant, T0=None, **over):
    res = []
    for search in (0, 1):
        prm = fr.params_default(variant, search=search, **over)
        res.append(fr.register(t, P, T0=T0, params=prm, trace_capacity=4000))
    return res


@pytest.mark.parametrize("variant", ["p2p", "p2p_welsch", "p2pl_welsch", "p2pl"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_tile_search_equals_query_search(fr, variant, precision):
    pair = synth.config_pair(2, 0.05)                 # M = 4000 (ragged last tile of 32), N = 5000
    t = fr.target_create(pair.Q, pair.normals)
    over = dict(precision=precision)
    if variant in ("p2p", "p2pl"):
        over["max_iters"] = 100
    a, b = _both(fr, t, pair.P, variant, **over)
    _same(a, b)


@pytest.mark.parametrize("cfg,scale,variant", [(1, 1.0, "p2p_welsch"), (3, 0.02, "p2pl_welsch"),
                                                (3, 0.02, "p2p_welsch")])
def test_tile_search_equals_query_search_other_surfaces(fr, cfg, scale, variant):
    pair = synth.config_pair(cfg, scale)
    t = fr.target_create(pair.Q, pair.normals)
    a, b = _both(fr, t, pair.P, variant)
    _same(a, b)


def test_tile_search_far_source_and_tiny_sets(fr):
    """A source moved several diagonals away: every warm-started tile reaches
    most of the target (the candidate list overflows and the tile falls back to
    per-query search). Also one-bucket and one-point targets and sources."""
    pair = synth.config_pair(2, 0.3)                  # N = 30000: more buckets than a list holds
    t = fr.target_create(pair.Q)
    T0 = np.eye(4)
    T0[:3, 3] = [4.0, -3.0, 2.5]
    a, b = _both(fr, t, pair.P, "p2p", T0=T0, max_iters=30)
    _same(a, b)
    g = np.random.default_rng(7)
    for N, M in ((1, 1), (5, 40), (16, 33), (17, 1000)):
        Q = g.random((N, 3)).astype(np.float32)
        P = (g.random((M, 3)) * 0.9 + 0.05).astype(np.float32)
        tt = fr.target_create(Q)
        a, b = _both(fr, tt, P, "p2p", max_iters=20)
        _same(a, b)


@pytest.mark.parametrize("cfg,variant", [(2, "p2p_welsch"), (3, "p2pl_welsch")])
def test_tile_search_equals_query_search_full_size(fr, cfg, variant):
    pair = synth.config_pair(cfg)
    t = fr.target_create(pair.Q, pair.normals)
    a, b = _both(fr, t, pair.P, variant)
    _same(a, b)
