"""Seeded synthetic point sets and query sets.

This module only draws random numbers.  It holds none of the k-d tree
arithmetic, so the CPU oracle and the CUDA library can both be fed from it
without sharing any of the method.  Every generator takes an explicit seed
and uses numpy's PCG64 generator, so a (recipe, size, seed) triple always
produces the same float32 arrays on every machine.

Recipes:
  * ``uniform``   points uniform in a box (the paper's test rig, Sec. 4, draws
                  uniform points in [0,1]^4).
  * ``gmm``       an isotropic Gaussian mixture with equal weights (clustered
                  data); ``gmm_queries`` mixes mixture draws with uniform ones.
  * ``surface``   points area-uniform on random spheres and tori, with
                  Gaussian jitter.
  * ``clouds``    many independent small mixtures of log-uniform size, for the
                  batched multi-tree path.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 221012859


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, D: int, lo: float = 0.0, hi: float = 1.0, seed: int = 0) -> np.ndarray:
    g = rng(seed)
    return (lo + (hi - lo) * g.random((n, D))).astype(np.float32)


@dataclass
class Mixture:
    centres: np.ndarray   # [C, D]
    sigmas: np.ndarray    # [C]


def gmm_mixture(n_comp: int = 64, D: int = 3, sigma: float = 0.01, seed: int = 0) -> Mixture:
    g = rng(seed)
    centres = g.random((n_comp, D))
    return Mixture(centres, np.full(n_comp, sigma))


def gmm_sample(mix: Mixture, n: int, seed: int) -> np.ndarray:
    """Equal-weight draws from the mixture (points are not clipped)."""
    g = rng(seed)
    comp = g.integers(0, len(mix.sigmas), size=n)
    pts = mix.centres[comp] + mix.sigmas[comp, None] * g.standard_normal((n, mix.centres.shape[1]))
    return pts.astype(np.float32)


def gmm_queries(mix: Mixture, n: int, frac_uniform: float, seed: int) -> np.ndarray:
    """A fraction ``frac_uniform`` uniform in [0,1]^D, the rest from the mixture."""
    g = rng(seed)
    D = mix.centres.shape[1]
    is_uni = g.random(n) < frac_uniform
    comp = g.integers(0, len(mix.sigmas), size=n)
    q = mix.centres[comp] + mix.sigmas[comp, None] * g.standard_normal((n, D))
    uni = g.random((n, D))
    q[is_uni] = uni[is_uni]
    return q.astype(np.float32)


def gmm_query_is_uniform(n: int, frac_uniform: float, seed: int) -> np.ndarray:
    """Which of the ``gmm_queries(mix, n, frac_uniform, seed)`` queries were drawn
    uniformly (the generator's first draw); those land between the clusters
    (the mixture covers a small part of the cube)."""
    return rng(seed).random(n) < frac_uniform


@dataclass
class Shapes:
    kind: np.ndarray      # [S] 0 = sphere, 1 = torus
    centre: np.ndarray    # [S, 3]
    R: np.ndarray         # [S] sphere radius or torus major radius
    r: np.ndarray         # [S] torus minor radius (unused for spheres)
    axis: np.ndarray      # [S, 3] torus axis (unit)
    area: np.ndarray      # [S]


def surface_shapes(n_shapes: int = 256, seed: int = 0) -> Shapes:
    g = rng(seed)
    kind = (g.random(n_shapes) < 0.5).astype(np.int64)
    centre = g.random((n_shapes, 3))
    R = 0.01 + 0.09 * g.random(n_shapes)
    r = R * (0.2 + 0.3 * g.random(n_shapes))
    ax = g.standard_normal((n_shapes, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    area = np.where(kind == 0, 4.0 * np.pi * R * R, 4.0 * np.pi * np.pi * R * r)
    return Shapes(kind, centre, R, r, ax, area)


def _frame(axis: np.ndarray):
    helper = np.where(np.abs(axis[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    e1 = np.cross(axis, helper)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(axis, e1)
    return e1, e2


def surface_sample(sh: Shapes, n: int, seed: int, jitter: float = 1e-4) -> np.ndarray:
    """Area-uniform points on the shapes (shape chosen with probability
    proportional to its area), plus N(0, jitter^2) per coordinate."""
    g = rng(seed)
    s = g.choice(len(sh.area), size=n, p=sh.area / sh.area.sum())
    out = np.empty((n, 3))
    sph = sh.kind[s] == 0
    # spheres: normalised Gaussian directions
    i_s = np.nonzero(sph)[0]
    v = g.standard_normal((len(i_s), 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    out[i_s] = sh.centre[s[i_s]] + sh.R[s[i_s], None] * v
    # tori: major angle uniform, minor angle by rejection with weight
    # (R + r cos v) / (R + r), which makes the points area-uniform
    i_t = np.nonzero(~sph)[0]
    st = s[i_t]
    R, r = sh.R[st], sh.r[st]
    u = 2.0 * np.pi * g.random(len(i_t))
    vv = np.empty(len(i_t))
    todo = np.arange(len(i_t))
    while len(todo):
        cand = 2.0 * np.pi * g.random(len(todo))
        acc = g.random(len(todo)) * (R[todo] + r[todo]) <= R[todo] + r[todo] * np.cos(cand)
        vv[todo[acc]] = cand[acc]
        todo = todo[~acc]
    rho = R + r * np.cos(vv)
    e1, e2 = _frame(sh.axis[st])
    out[i_t] = (sh.centre[st] + (rho * np.cos(u))[:, None] * e1 + (rho * np.sin(u))[:, None] * e2
                + (r * np.sin(vv))[:, None] * sh.axis[st])
    out += jitter * g.standard_normal((n, 3))
    return out.astype(np.float32)


@dataclass
class Clouds:
    points: np.ndarray     # [sum N_i, 3]
    offsets: np.ndarray    # [T+1] int64
    queries: np.ndarray    # [sum Q_i, 3]
    qoffsets: np.ndarray   # [T+1] int64


def clouds(T: int, log2_min: float = 8.0, log2_max: float = 18.0, seed: int = 0,
           sigma_lo: float = 0.005, sigma_hi: float = 0.05, max_comp: int = 8) -> Clouds:
    """T independent 3-D clouds: N_i = round(2^U[log2_min, log2_max]); each a
    mixture of 1..max_comp equal-weight isotropic Gaussians with centres
    uniform in [0,1]^3 and sigma log-uniform in [sigma_lo, sigma_hi];
    Q_i = N_i queries from the same mixture."""
    g = rng(seed)
    sizes = np.rint(2.0 ** g.uniform(log2_min, log2_max, size=T)).astype(np.int64)
    offsets = np.zeros(T + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    total = int(offsets[-1])
    pts = np.empty((total, 3), dtype=np.float32)
    qs = np.empty((total, 3), dtype=np.float32)
    for t in range(T):
        C = int(g.integers(1, max_comp + 1))
        centres = g.random((C, 3))
        sig = np.exp(g.uniform(np.log(sigma_lo), np.log(sigma_hi), size=C))
        n = int(sizes[t])
        for dst in (pts, qs):
            comp = g.integers(0, C, size=n)
            dst[offsets[t]:offsets[t + 1]] = (centres[comp] + sig[comp, None] * g.standard_normal((n, 3)))
    return Clouds(pts, offsets, qs, offsets.copy())


# --------------------------------------------------------------------------
# Named workloads.  ``seed = BASE_SEED + workload number``.
# --------------------------------------------------------------------------

def uniform_small(n: int = 1 << 14, q: int = 1 << 14, seed: int = BASE_SEED + 1):
    """N uniform in [0,1]^3, Q queries uniform in [-0.1, 1.1]^3."""
    return uniform(n, 3, 0.0, 1.0, seed), uniform(q, 3, -0.1, 1.1, seed + 1000)


def gmm_large(n: int = 1 << 24, q: int = 1 << 24, seed: int = BASE_SEED + 2):
    """64-component mixture, sigma 0.01, centres U[0,1]^3; queries 90% mixture,
    10% uniform in [0,1]^3."""
    mix = gmm_mixture(64, 3, 0.01, seed)
    return gmm_sample(mix, n, seed + 1), gmm_queries(mix, q, 0.1, seed + 2)


def surface_set(n: int, q: int, seed: int = BASE_SEED + 3, q_seed_offset: int = 2):
    """Points and queries from the same 256 spheres / tori."""
    sh = surface_shapes(256, seed)
    return surface_sample(sh, n, seed + 1), surface_sample(sh, q, seed + q_seed_offset)


def uniform_dim(n: int, q: int, D: int, seed: int = BASE_SEED + 3):
    return uniform(n, D, 0.0, 1.0, seed + 10 * D), uniform(q, D, 0.0, 1.0, seed + 10 * D + 1)
