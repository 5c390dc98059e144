"""Seeded synthetic point-set pairs shaped like the scans of the paper's experiments.

This module holds none of the registration method's arithmetic. It samples
surfaces (torus, sum-of-Gaussian-bumps height field, union of ellipsoids),
crops a pair to a stated overlap with two parallel half-spaces, adds Gaussian
noise and uniform outliers the way the paper's synthetic tests do (crops,
noise and uniform outliers: Sec. 6.1, Fig. 5), and moves the source by a
seeded rigid motion. Both the CUDA path and the FP64 oracle consume exactly the
float32 arrays produced here; nothing here depends on either of them.

Random numbers come from numpy's Philox counter-based generator (Salmon et al.,
SC'11), keyed by the seed, so every pair is reproducible from its seed alone.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial.transform import Rotation

__all__ = [
    "Pair", "rng", "random_rigid", "torus_pair", "height_field_pair",
    "ellipsoid_pair", "config_pair", "CONFIG_SEEDS", "BATCH_VARIANTS", "batch_specs", "make_pair",
    "batch_pairs", "serve_specs", "serve_requests", "rotation_about", "robustness_starts",
]

# Seed of workload i (1-based) is 20070762 + i.
CONFIG_SEEDS = {i: 20070762 + i for i in range(1, 6)}


@dataclasses.dataclass
class Pair:
    """One registration problem: align source P onto target Q.

    P, Q: float32 [M,3], [N,3]. normals: float32 [N,3] unit normals of Q (or None).
    R_gt, t_gt: float64 ground-truth motion taking P onto Q (x -> R_gt x + t_gt).
    diag: bounding-box diagonal of the clean target surface.
    src_normals: float32 [M,3] unit normals of P: the surface normal at each sampled
    point moved with the source (noise moves positions only); an outlier gets a
    random unit normal.
    """
    P: np.ndarray
    Q: np.ndarray
    normals: np.ndarray | None
    R_gt: np.ndarray
    t_gt: np.ndarray
    diag: float
    name: str = ""
    src_normals: np.ndarray | None = None

    @property
    def M(self) -> int:
        return int(self.P.shape[0])

    @property
    def N(self) -> int:
        return int(self.Q.shape[0])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def random_rigid(g: np.random.Generator, max_angle_deg: float, max_trans: float):
    """Axis uniform on S^2, angle uniform in [0, max_angle], translation uniform per axis."""
    axis = g.standard_normal(3)
    axis /= np.linalg.norm(axis)
    angle = math.radians(max_angle_deg) * g.random()
    R = Rotation.from_rotvec(axis * angle).as_matrix()
    t = (2.0 * g.random(3) - 1.0) * max_trans
    return R, t


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


# ----------------------------------------------------------------------------
# Surfaces. Each sampler draws area-uniform points (rejection on the area
# element) restricted to a region given by `keep(points) -> bool mask`.
# ----------------------------------------------------------------------------

def _fill(draw, n: int, keep, g: np.random.Generator):
    pts, nrm, have = [], [], 0
    while have < n:
        x, nx = draw(max(4096, 2 * (n - have)))
        if keep is not None:
            mk = keep(x)
            x, nx = x[mk], nx[mk]
        pts.append(x)
        nrm.append(nx)
        have += x.shape[0]
    return np.concatenate(pts)[:n], np.concatenate(nrm)[:n]


def _torus_draw(g, R=1.0, r=0.4):
    def draw(n):
        th = 2 * math.pi * g.random(n)
        ph = 2 * math.pi * g.random(n)
        acc = g.random(n) * (R + r) <= (R + r * np.cos(ph))
        th, ph = th[acc], ph[acc]
        ring = R + r * np.cos(ph)
        x = np.stack([ring * np.cos(th), ring * np.sin(th), r * np.sin(ph)], 1)
        nx = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], 1)
        return x, nx
    return draw


def _height_params(g, bumps=16):
    return dict(a=g.uniform(-0.15, 0.15, bumps), s=g.uniform(0.05, 0.2, bumps),
                c=g.random((bumps, 2)))


def _height_eval(hp, xy):
    d = xy[:, None, :] - hp["c"][None]                      # [n,k,2]
    e = hp["a"] * np.exp(-(d ** 2).sum(-1) / (2 * hp["s"] ** 2))   # [n,k]
    z = e.sum(1)
    grad = -(e[..., None] * d / (hp["s"] ** 2)[None, :, None]).sum(1)   # [n,2]
    return z, grad


def _height_draw(g, hp):
    gx = np.linspace(0, 1, 161)
    xy = np.stack(np.meshgrid(gx, gx), -1).reshape(-1, 2)
    _, gr = _height_eval(hp, xy)
    amax = 1.1 * np.sqrt(1 + (gr ** 2).sum(1)).max()

    def draw(n):
        xy = g.random((n, 2))
        z, gr = _height_eval(hp, xy)
        area = np.sqrt(1 + (gr ** 2).sum(1))
        acc = g.random(n) * amax <= area
        xy, z, gr = xy[acc], z[acc], gr[acc]
        x = np.concatenate([xy, z[:, None]], 1)
        nx = _unit(np.concatenate([-gr, np.ones((gr.shape[0], 1))], 1))
        return x, nx
    return draw


def _ellipsoid_params(g, count=8):
    cen = g.random((count, 3))
    ax = g.uniform(0.1, 0.3, (count, 3))
    rot = Rotation.random(count, random_state=g).as_matrix()
    # quadratic form of ellipsoid k: (x-c)^T A_k (x-c) = 1
    A = np.einsum("kij,kj,klj->kil", rot, 1.0 / ax ** 2, rot)
    p = 1.6075   # Knud Thomsen's surface-area approximation, used only as sampling weights
    a, b, c = ax[:, 0], ax[:, 1], ax[:, 2]
    area = 4 * math.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p)
    return dict(c=cen, ax=ax, rot=rot, A=A, w=area / area.sum())


def _ellipsoid_draw(g, ep):
    cnt = ep["c"].shape[0]

    def draw(n):
        k = g.choice(cnt, size=n, p=ep["w"])
        u = _unit(g.standard_normal((n, 3)))
        ax = ep["ax"][k]
        dens = np.linalg.norm(u / ax, axis=1) * ax.min(1)
        acc = g.random(n) <= dens
        k, u, ax = k[acc], u[acc], ax[acc]
        x = ep["c"][k] + np.einsum("nij,nj->ni", ep["rot"][k], ax * u)
        nx = _unit(np.einsum("nij,nj->ni", ep["A"][k], x - ep["c"][k]))
        # keep only the outer surface of the union
        d = x[:, None, :] - ep["c"][None]
        inside = np.einsum("nki,kij,nkj->nk", d, ep["A"], d) < 1.0
        inside[np.arange(k.size), k] = False
        ok = ~inside.any(1)
        return x[ok], nx[ok]
    return draw


# ----------------------------------------------------------------------------
# Pair assembly
# ----------------------------------------------------------------------------

def _crop_bounds(g, draw, overlap: float, dim: int, pool: int = 200_000):
    """Two parallel half-spaces with `overlap` of the source inside the target's.

    Target keeps a.x >= s_T, source keeps a.x <= s_S; quantiles chosen so the
    target and source regions cover the same share of the surface.
    """
    if overlap >= 1.0:
        return None, None
    a = _unit(g.standard_normal(dim))
    sample, _ = draw(pool)
    v = sample[:, :dim] @ a
    fs = 1.0 / (2.0 - overlap)
    s_T = float(np.quantile(v, 1.0 - fs))
    s_S = float(np.quantile(v, fs))
    keep_T = lambda x: x[:, :dim] @ a >= s_T
    keep_S = lambda x: x[:, :dim] @ a <= s_S
    return keep_T, keep_S


def _assemble(g, draw, M, N, overlap, noise, outliers, max_angle, dim_crop, name, pool=200_000):
    keep_T, keep_S = _crop_bounds(g, draw, overlap, dim_crop, pool)
    Q, nQ = _fill(draw, N, keep_T, g)
    diag = float(np.linalg.norm(Q.max(0) - Q.min(0)))
    n_out = int(round(outliers * M))
    S, nS = _fill(draw, M - n_out, keep_S, g)
    S = S + noise * diag * g.standard_normal(S.shape)
    if n_out:
        lo, hi = S.min(0), S.max(0)
        S = np.concatenate([S, lo + (hi - lo) * g.random((n_out, 3))])
        nS = np.concatenate([nS, np.zeros((n_out, 3))])
    perm = g.permutation(S.shape[0])
    S, nS = S[perm], nS[perm]
    R_s, t_s = random_rigid(g, max_angle, 0.1 * diag)
    P = S @ R_s.T + t_s
    if n_out:   # drawn after everything above, so P and Q do not depend on it
        out = perm >= M - n_out
        nS[out] = _unit(g.standard_normal((int(out.sum()), 3)))
    nP = nS @ R_s.T
    return Pair(P=P.astype(np.float32), Q=Q.astype(np.float32),
                normals=nQ.astype(np.float32), R_gt=R_s.T.copy(),
                t_gt=-(R_s.T @ t_s), diag=diag, name=name, src_normals=nP.astype(np.float32))


def torus_pair(seed, M=2000, N=2000, overlap=1.0, noise=0.002, outliers=0.0,
               max_angle=30.0, crop_pool=200_000) -> Pair:
    g = rng(seed)
    return _assemble(g, _torus_draw(g), M, N, overlap, noise, outliers, max_angle,
                     3, "torus", crop_pool)


def height_field_pair(seed, M=80_000, N=100_000, overlap=0.6, noise=0.005,
                      outliers=0.10, max_angle=25.0, crop_pool=200_000) -> Pair:
    g = rng(seed)
    hp = _height_params(g)
    return _assemble(g, _height_draw(g, hp), M, N, overlap, noise, outliers,
                     max_angle, 2, "height_field", crop_pool)


def ellipsoid_pair(seed, M=200_000, N=500_000, overlap=0.5, noise=0.003,
                   outliers=0.05, max_angle=25.0, crop_pool=200_000) -> Pair:
    g = rng(seed)
    ep = _ellipsoid_params(g)
    return _assemble(g, _ellipsoid_draw(g, ep), M, N, overlap, noise, outliers,
                     max_angle, 3, "ellipsoids", crop_pool)


def config_pair(i: int, scale: float = 1.0) -> Pair:
    """The single-pair workloads 1-3 (optionally with M, N scaled down for tests)."""
    s = CONFIG_SEEDS[i]
    if i == 1:
        return torus_pair(s, M=max(8, int(2000 * scale)), N=max(8, int(2000 * scale)))
    if i == 2:
        return height_field_pair(s, M=max(8, int(80_000 * scale)), N=max(8, int(100_000 * scale)))
    if i == 3:
        return ellipsoid_pair(s, M=max(8, int(200_000 * scale)), N=max(8, int(500_000 * scale)))
    raise ValueError(f"no single-pair workload {i}")


# ----------------------------------------------------------------------------
# Many-pair workloads
# ----------------------------------------------------------------------------

BATCH_VARIANTS = ("p2p", "p2p_welsch", "p2pl_welsch")
_GENERATORS = (torus_pair, height_field_pair, ellipsoid_pair)


def _log_uniform(g, lo, hi) -> float:
    return math.exp(g.uniform(math.log(lo), math.log(hi)))


def batch_specs(seed: int = CONFIG_SEEDS[4], npairs: int = 256, lo: int = 2000, hi: int = 200_000,
                variants=BATCH_VARIANTS) -> list:
    """Per-pair recipe of a mixed batch (cheap; make_pair builds one pair):
    M and N each log-uniform in [lo, hi], variants cycled in equal shares,
    surface generator uniform over torus / height field / ellipsoids, overlap
    U[0.5, 1], outliers U[0, 0.1], rotation angle up to 30 degrees, and a
    sub-seed per pair."""
    g = rng(seed)
    out = []
    for k in range(npairs):
        M = int(round(_log_uniform(g, lo, hi)))
        N = int(round(_log_uniform(g, lo, hi)))
        kind = int(g.integers(3))
        overlap = float(g.uniform(0.5, 1.0))
        outliers = float(g.uniform(0.0, 0.1))
        sub_seed = int(g.integers(1 << 62))
        out.append(dict(variant=variants[k % len(variants)], kind=kind, M=M, N=N, overlap=overlap,
                        outliers=outliers, seed=sub_seed))
    return out


def make_pair(spec: dict):
    """(variant, Pair) of one batch_specs entry (the crop planes come from a
    sample of max(20000, M + N) surface points)."""
    M, N = spec["M"], spec["N"]
    pair = _GENERATORS[spec["kind"]](spec["seed"], M=M, N=N, overlap=spec["overlap"], outliers=spec["outliers"],
                                     max_angle=30.0, crop_pool=max(20_000, M + N))
    return spec["variant"], pair


def batch_pairs(seed: int = CONFIG_SEEDS[4], npairs: int = 256, lo: int = 2000, hi: int = 200_000,
                variants=BATCH_VARIANTS) -> list:
    """Mixed batch of independent registrations (batch_specs, then make_pair
    for each). Returns a list of (variant, Pair)."""
    return [make_pair(s) for s in batch_specs(seed, npairs, lo, hi, variants)]


SERVE_VARIANTS = ("p2p_welsch", "p2pl_welsch")


def serve_specs(seed: int = CONFIG_SEEDS[5], n: int = 64, lo: int = 1000, hi: int = 1_000_000) -> list:
    """Recipes of serving-workload requests: robust registrations (Welsch
    point-to-point and point-to-plane, alternating), M and N log-uniform in
    [lo, hi], the same surface generators, overlap U[0.5, 1], outliers
    U[0, 0.1]; arrival times are drawn by the caller from the rate it sweeps."""
    return batch_specs(seed, n, lo, hi, variants=SERVE_VARIANTS)


def serve_requests(seed: int = CONFIG_SEEDS[5], n: int = 64, lo: int = 1000, hi: int = 1_000_000) -> list:
    """serve_specs built into (variant, Pair) requests."""
    return [make_pair(s) for s in serve_specs(seed, n, lo, hi)]


# ----------------------------------------------------------------------------
# Random initial alignments (Sec. 6.4 limitations experiment)
# ----------------------------------------------------------------------------

def rotation_about(axis, angle_rad: float, centre) -> np.ndarray:
    """4x4 rotation by `angle_rad` about the unit `axis` through `centre`."""
    a = np.asarray(axis, dtype=np.float64)
    R = Rotation.from_rotvec(a / np.linalg.norm(a) * angle_rad).as_matrix()
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = np.asarray(centre, np.float64) - R @ np.asarray(centre, np.float64)
    return T


def robustness_starts(pair: Pair, angles_deg=(5, 10, 20, 30, 50), per_angle: int = 10, seed: int = 20070770):
    """Initial transforms that rotate the source from its ground-truth position
    by a fixed angle about a random axis (uniform on the sphere) through the
    aligned source's centroid, `per_angle` axes per angle. Returns a list of
    (angle_deg, T0) with T0 = Rot o T_gt (x -> R_gt x + t_gt first)."""
    g = rng(seed)
    T_gt = np.eye(4)
    T_gt[:3, :3] = pair.R_gt
    T_gt[:3, 3] = pair.t_gt
    centre = (pair.P.astype(np.float64) @ pair.R_gt.T + pair.t_gt).mean(axis=0)
    out = []
    for ang in angles_deg:
        for _ in range(per_angle):
            out.append((ang, rotation_about(_unit(g.standard_normal(3)), math.radians(ang), centre) @ T_gt))
    return out
