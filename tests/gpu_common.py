"""Shared helpers of the GPU parity tests: the parity bars and oracle-side
single-pass quantities built from oracle primitives."""
import math

import numpy as np

import oracle

# Parity bars (closest point: exact index or a near tie; transform tolerances).
NN_TIE_REL = 1e-6
R_TOL_RAD = 1e-5
T_TOL_DIAG = 1e-6


def assert_nn_parity(idx_g, d2_g, idx_o, d2_o, d2s_o):
    """Indices equal, except where the oracle's best and second-best squared
    distances differ by under 1e-6 relative; there the distances agree to 1e-6."""
    idx_g = np.asarray(idx_g)
    d2_g = np.asarray(d2_g)
    same = idx_g == idx_o
    tie = (d2s_o - d2_o) < NN_TIE_REL * d2s_o
    bad = ~same & ~tie
    assert not bad.any(), f"{bad.sum()} index mismatches outside the tie rule, e.g. {np.flatnonzero(bad)[:5]}"
    diff = ~same
    if diff.any():
        rel = np.abs(d2_g[diff] - d2_o[diff]) / np.maximum(d2_o[diff], 1e-300)
        assert (rel <= NN_TIE_REL).all(), rel.max()
    # same index: both FP64, from the same FP32 point; only rounding differs
    rel = np.abs(d2_g[same] - d2_o[same]) / np.maximum(d2_o[same], 1e-30)
    assert (rel <= 1e-9).all(), rel.max()
    return int(diff.sum())


def rotation_angle(Ra, Rb) -> float:
    c = (np.trace(Ra @ Rb.T) - 1.0) / 2.0
    return math.acos(max(-1.0, min(1.0, c)))


def random_T(g, max_angle, max_t):
    from scipy.spatial.transform import Rotation
    ax = g.standard_normal(3)
    ax /= np.linalg.norm(ax)
    T = np.eye(4)
    T[:3, :3] = Rotation.from_rotvec(ax * max_angle * g.random()).as_matrix()
    T[:3, 3] = (2 * g.random(3) - 1) * max_t
    return T


def oracle_pass_p2p(P32, Q32, Tn, nu, scale, center, robust):
    """Energy and T' of one Alg. 1 pass at the normalised transform Tn."""
    nz = oracle.Normalization(c=np.asarray(center, float), s=scale)
    Pn, Qn = nz.fwd(np.asarray(P32, float)), nz.fwd(np.asarray(Q32, float))
    idx, d2, _ = oracle.closest(oracle.apply(Tn, Pn), Qn)
    if robust:
        E = float(oracle.welsch(np.sqrt(d2), nu).sum())
        w = np.exp(-d2 / (2 * nu * nu))
    else:
        E = float(d2.sum())
        w = np.ones_like(d2)
    return E, oracle.weighted_procrustes(Pn, Qn[idx], w)


def oracle_pass_p2pl(P32, Q32, N32, Tn, nu, scale, center):
    """Energy and xi* = G_ppl(xi) of one Alg. 2 pass at xi = log(Tn)."""
    nz = oracle.Normalization(c=np.asarray(center, float), s=scale)
    Pn, Qn = nz.fwd(np.asarray(P32, float)), nz.fwd(np.asarray(Q32, float))
    Nr = np.asarray(N32, float)
    xi = oracle.se3_vee(oracle.se3_log(Tn))
    T = oracle.se3_transform(xi)
    X = oracle.apply(T, Pn)
    idx, _, _ = oracle.closest(X, Qn)
    n = Nr[idx]
    B = np.einsum("nd,nd->n", X - Qn[idx], n)
    E = float(oracle.welsch(B, nu).sum())
    gamma = np.exp(-B ** 2 / (2 * nu * nu))
    J = oracle.plane_gradient(xi, Pn, n)
    A = (J * gamma[:, None]).T @ J
    b = (J * gamma[:, None]).T @ (J @ xi - B)
    return E, np.linalg.solve(A, b), xi
