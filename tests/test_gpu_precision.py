"""Precision variants (fricp_params.precision) against the FP64 oracle.

FP64 is the reference mode (exact FP64 argmin, FP64 per-point terms; all other
GPU parity tests run in it). FP32 computes the transform, distances and weights
in float and FP16 storage also quantises the target coordinates to 16-bit
offsets in their bucket's box; both keep the sums and solves in FP64. On
registrations the oracle itself holds stable, their error against the oracle is
bounded here (about 20x the largest error measured on GB300 when the bounds were
set); on chaotic ones they follow their own trajectory, like any other rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2007_07627_gb300 import synth
from tests.gpu_common import rotation_angle

pytestmark = pytest.mark.gpu

S = synth.CONFIG_SEEDS
# (name, pair, variant, overrides, {precision: (max rad, max t / diag, max rel. energy)})
CASES = [
    ("torus_fast_icp", lambda: synth.config_pair(1), "p2p", {"max_iters": 100},
     {"fp32": (1e-6, 1e-6, 1e-6), "fp16": (3e-3, 2e-3, 2e-3)}),
    ("ellipsoids_full_p2pl", lambda: synth.ellipsoid_pair(S[3], M=4000, N=10000, overlap=1.0, outliers=0.0),
     "p2pl_welsch", {}, {"fp32": (2e-3, 5e-4, 2e-3), "fp16": (7e-3, 1e-3, 2e-2)}),
]


@pytest.fixture(scope="module")
def fr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2007_07627_gb300 import build
    build.build()
    import paper_2007_07627_gb300 as fr
    fr.lib()
    return fr


@pytest.mark.parametrize("name,make,variant,over,bounds", CASES, ids=[c[0] for c in CASES])
def test_reduced_precision_error_against_oracle(fr, name, make, variant, over, bounds):
    pair = make()
    o = oracle.register(pair.P, pair.Q, oracle.Params(variant=variant, **over), normals=pair.normals)
    t = fr.target_create(pair.Q, pair.normals)
    ref = fr.register(t, pair.P, params=fr.params_default(variant, **over))
    assert ref["iterations"] == o["iterations"]          # the reference mode, exact on these cases
    for prec, (ang, tr, en) in bounds.items():
        r = fr.register(t, pair.P, params=fr.params_default(variant, precision=prec, **over))
        assert r["status"] == "OK"
        assert rotation_angle(r["R"], o["R"]) < ang, (prec, rotation_angle(r["R"], o["R"]))
        assert np.abs(r["t"] - o["t"]).max() < tr * pair.diag, prec
        assert abs(r["final_energy"] - o["final_energy"]) <= en * abs(o["final_energy"]), prec
    t.destroy()


def test_fp64_mode_is_the_default(fr):
    pair = synth.config_pair(3, 0.01)
    t = fr.target_create(pair.Q, pair.normals)
    a = fr.register(t, pair.P, params=fr.params_default("p2pl_welsch"))
    b = fr.register(t, pair.P, params=fr.params_default("p2pl_welsch", precision="fp64"))
    assert np.array_equal(a["R"], b["R"]) and a["iterations"] == b["iterations"]
    t.destroy()


def test_mixed_precision_batch_equals_alone(fr):
    batch = synth.batch_pairs(seed=99, npairs=6, lo=500, hi=4000)
    precs = ["fp64", "fp32", "fp16", "fp32", "fp16", "fp64"]
    targets = [fr.target_create(p.Q, p.normals) for _, p in batch]
    prms = [fr.params_default(v, precision=pr, **({"max_iters": 100} if v == "p2p" else {}))
            for (v, _), pr in zip(batch, precs)]
    res = fr.batch_register(targets, [p.P for _, p in batch], prms)
    for k in range(len(batch)):
        alone = fr.register(targets[k], batch[k][1].P, params=prms[k])
        assert res[k]["iterations"] == alone["iterations"], k
        assert np.array_equal(res[k]["R"], alone["R"]) and np.array_equal(res[k]["t"], alone["t"]), k
    for t in targets:
        t.destroy()


def test_fp16_storage_quantisation_is_bounded(fr):
    """Closest points found on FP16-stored targets, returned through a whole
    registration's last correspondence, stay within the quantisation of the
    bucket boxes: the run ends near the FP64 run on an exact copy."""
    g = np.random.default_rng(7)
    Q = (g.random((20000, 3)) * [1.0, 1.0, 0.2]).astype(np.float32)
    t = fr.target_create(Q)
    r = fr.register(t, Q, params=fr.params_default("p2p", precision="fp16", max_iters=100))
    assert rotation_angle(r["R"], np.eye(3)) < 1e-3 and np.abs(r["t"]).max() < 1e-3
    t.destroy()


def test_invalid_precision_is_rejected(fr):
    pair = synth.config_pair(1, 0.1)
    t = fr.target_create(pair.Q)
    with pytest.raises(fr.FricpError):
        fr.register(t, pair.P, params=fr.params_default("p2p", precision=7))
    t.destroy()
