"""Random initial alignments as a batched workload (the limitations experiment
of Sec. 6: the source rotated from its ground-truth position by a fixed angle
about a random axis) and the nu schedule comparison of Sec. 4.3 (Fig. 4).

Checks: the batched sweep equals the one-at-a-time runs bit for bit, one
rotated start against the oracle, and the method's documented behaviour on a
pair with 50% outliers (robust solvers beat the plain one; a decreasing nu
beats a fixed nu_min).
"""
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


@pytest.fixture(scope="module")
def pair():
    return synth.ellipsoid_pair(synth.CONFIG_SEEDS[3] + 100, M=4000, N=4000, overlap=1.0, noise=0.003,
                                outliers=0.5, max_angle=0.0)


def _rmse(P, R, t, R_gt, t_gt):
    d = P.astype(np.float64) @ (R_gt - R).T + (t_gt - t)
    return float(np.sqrt((d * d).sum(axis=1).mean()))


def test_rotated_starts_are_what_they_say(pair):
    for ang, T0 in synth.robustness_starts(pair, angles_deg=(5, 30), per_angle=3):
        R_rel = T0[:3, :3] @ pair.R_gt.T
        got = np.degrees(np.arccos(np.clip((np.trace(R_rel) - 1) / 2, -1, 1)))
        assert abs(got - ang) < 1e-9


def test_sweep_batched_equals_alone_and_robust_solvers_win(fr, pair):
    starts = synth.robustness_starts(pair, angles_deg=(5, 30), per_angle=2)
    variants = ("p2p", "p2p_welsch", "p2pl_welsch")
    cases = [(v, T0) for v in variants for _, T0 in starts]
    t = fr.target_create(pair.Q, pair.normals)
    prms = [fr.params_default(v) for v, _ in cases]
    res = fr.batch_register([t] * len(cases), [pair.P] * len(cases), prms, T0=np.stack([T0 for _, T0 in cases]))
    err = {}
    for (v, T0), prm, r in zip(cases, prms, res):
        a = fr.register(t, pair.P, T0=T0, params=prm)
        assert a["iterations"] == r["iterations"] and np.array_equal(a["R"], r["R"]) and np.array_equal(a["t"], r["t"])
        err.setdefault(v, []).append(_rmse(pair.P, r["R"], r["t"], pair.R_gt, pair.t_gt) / pair.diag)
    assert max(err["p2p_welsch"]) < 0.5 * min(err["p2p"])
    assert max(err["p2pl_welsch"]) < 0.5 * min(err["p2p"])
    t.destroy()


def test_rotated_start_matches_oracle(fr, pair):
    ang, T0 = synth.robustness_starts(pair, angles_deg=(30,), per_angle=1)[0]
    t = fr.target_create(pair.Q, pair.normals)
    r = fr.register(t, pair.P, T0=T0, params=fr.params_default("p2pl_welsch"), trace_capacity=4096)
    ref = oracle_reference(pair, "p2pl_welsch", {}, perms=(1, 2, 3, 4), jitters=4, T0=T0)
    assert_registration_parity(r, ref, pair.diag)
    t.destroy()


def test_decreasing_nu_beats_fixed_nu_min(fr, pair):
    """Fig. 4's comparison: a fixed nu = nu_min leaves too few weighted pairs."""
    T0 = synth.robustness_starts(pair, angles_deg=(10,), per_angle=1)[0][1]
    t = fr.target_create(pair.Q)
    dyn = fr.register(t, pair.P, T0=T0, params=fr.params_default("p2p_welsch"))
    lo = fr.register(t, pair.P, T0=T0, params=fr.params_default("p2p_welsch", nu_max=dyn["nu_min"],
                                                                nu_min=dyn["nu_min"]))
    e_dyn = _rmse(pair.P, dyn["R"], dyn["t"], pair.R_gt, pair.t_gt)
    e_lo = _rmse(pair.P, lo["R"], lo["t"], pair.R_gt, pair.t_gt)
    assert e_dyn < e_lo
    t.destroy()
