"""The parameter values the paper prints (tests/golden/paper_parameters.txt,
each line with its section) against the defaults of the oracle and of the C ABI
(fricp_params_default; a host call, no GPU) and against the oracle's nu rules."""
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "paper_parameters.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


G = _golden()


def test_fixture_is_complete_and_consistent():
    for k in ("anderson_m", "eps", "max_iters", "p2pl_iters_first", "p2pl_iters_cap", "nu_max_factor",
              "nu_min_divisor_p2p", "nu_min_divisor_p2pl", "nu_min_neighbours", "normal_neighbours", "nu_halving"):
        assert k in G, k
    assert G["nu_min_divisor_p2p"] == pytest.approx(3.0 * math.sqrt(3.0), rel=1e-15)


def test_oracle_defaults_are_the_papers():
    p = oracle.Params()
    assert p.anderson_m == G["anderson_m"] and p.eps == G["eps"] and p.max_iters == G["max_iters"]
    assert p.p2pl_iters_first == G["p2pl_iters_first"] and p.p2pl_iters_cap == G["p2pl_iters_cap"]


@pytest.mark.parametrize("variant", ["p2p", "p2p_welsch", "p2pl_welsch", "p2pl"])
def test_c_abi_defaults_are_the_papers(variant):
    from paper_2007_07627_gb300 import build
    build.build()
    import paper_2007_07627_gb300 as fr
    p = fr.params_default(variant)
    assert p.anderson_m == G["anderson_m"] and p.eps == G["eps"]
    assert p.nu_max <= 0.0 and p.nu_min <= 0.0   # the paper's rules, not fixed values
    if variant.startswith("p2pl"):
        if variant == "p2pl_welsch":
            assert p.p2pl_iters_first == G["p2pl_iters_first"] and p.p2pl_iters_cap == G["p2pl_iters_cap"]
    elif variant == "p2p_welsch":
        assert p.max_iters == G["max_iters"]


def test_oracle_nu_rules_use_the_printed_constants():
    # square grid of spacing h in z = 0: every interior point's six nearest distances
    # are h, h, h, h, h sqrt 2, h sqrt 2, so E_Q = h; in-plane normals give H_Q = 0
    h = 0.01
    xy = np.stack(np.meshgrid(np.arange(40) * h, np.arange(40) * h), -1).reshape(-1, 2)
    Q = np.column_stack([xy, np.zeros(len(xy))])
    assert oracle.nu_min_point_to_point(Q) == pytest.approx(h / G["nu_min_divisor_p2p"], rel=1e-12)
    # tilted normals: |(q_j - q) . n| = distance x sin(a) for the grid directions along x
    a = 0.3
    N = np.tile([math.sin(a), 0.0, math.cos(a)], (len(Q), 1))
    _, d2 = oracle.knn_self(Q, int(G["nu_min_neighbours"]))
    idx, _ = oracle.knn_self(Q, int(G["nu_min_neighbours"]))
    hq = np.median(np.median(np.abs(np.einsum("nkd,nd->nk", Q[idx] - Q[:, None, :], N)), axis=1))
    assert oracle.nu_min_point_to_plane(Q, N) == pytest.approx(hq / G["nu_min_divisor_p2pl"], rel=1e-12)


def test_oracle_nu_max_is_three_medians_and_stages_halve():
    """nu_max = 3 x the median initial distance (Sec. 4.3), in normalised units,
    and the stages run nu_max, nu_max / 2, ... down to nu_min (Sec. 4.3)."""
    g = np.random.default_rng(5)
    Q32 = g.random((400, 3)).astype(np.float32)
    P32 = (Q32 + 0.02 * g.standard_normal((400, 3))).astype(np.float32)[:300]
    P, Q = P32.astype(np.float64), Q32.astype(np.float64)
    nz = oracle.normalization(P, Q)
    r = oracle.register(P32, Q32, oracle.Params(variant="p2p_welsch", max_iters=3))
    med = float(np.median(np.sqrt(oracle.closest((P - nz.c) * nz.s, (Q - nz.c) * nz.s)[1])))
    assert r["nu_max"] == pytest.approx(G["nu_max_factor"] * med, rel=1e-9)
    stages = math.ceil(math.log(r["nu_max"] / r["nu_min"]) / math.log(1.0 / G["nu_halving"])) + 1
    assert r["stages"] == stages
