"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module only draws random numbers: point clouds, strengths and system
sizes.  It holds none of the Spectral Ewald arithmetic, so both the CUDA path
and the CPU oracle may take their inputs from here without sharing any of the
method's code.

The paper's experiments use uniformly distributed random points in a cube with
random source strengths (Section 9, "Results"); there is no dataset.  The
recipes below follow the workload descriptions of the five evaluated
configurations:

* ``uniform``   : x ~ U[x0, x0+L)^3, f ~ N(0, 1)^3
* ``blobs``     : 16 Gaussian blobs (sigma = 0.05, centres ~ U[0,1)^3) holding
                  80 % of the points plus a 20 % uniform background, points
                  redrawn until they fall in [0, 1)^3; f ~ N(0,1)^3 and q a
                  random unit vector per point
* ``batched``   : 64 systems, sizes lognormal(ln 1e4, 1) clipped to
                  [1e3, 1e5], 8 right-hand sides per system.

Every generator is a pure function of ``seed``: PCG64 seeded with
``SEED_BASE + seed``.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 160704808


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + int(seed), int(stream)]))


def uniform_points(n: int, seed: int, L=1.0, x0=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n points iid uniform in the half-open box [x0, x0+L), float64 (n, 3);
    L is one side (a cube) or three sides (Lx, Ly, Lz)."""
    x = _rng(seed, 1).random((n, 3)) * L + np.asarray(x0, dtype=np.float64)
    # random() is in [0, 1); scaling can round up to exactly x0+L, keep it half-open
    top = np.nextafter(np.asarray(x0, dtype=np.float64) + L, -np.inf)
    return np.minimum(x, top)


def normal_vectors(n: int, seed: int, comps: int = 3) -> np.ndarray:
    """n iid N(0, 1)^comps vectors, float64 (n, comps)."""
    return _rng(seed, 2).standard_normal((n, comps))


def uniform_vectors(n: int, seed: int, comps: int = 3) -> np.ndarray:
    """n vectors with iid U[-1, 1] components (the paper's strength recipe)."""
    return _rng(seed, 3).uniform(-1.0, 1.0, (n, comps))


def unit_vectors(n: int, seed: int) -> np.ndarray:
    """n random unit vectors (normalised Gaussian draws), float64 (n, 3)."""
    v = _rng(seed, 4).standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def blob_points(n: int, seed: int, n_centres: int = 16, sigma: float = 0.05,
                frac_background: float = 0.2) -> np.ndarray:
    """Clustered cloud in [0, 1)^3: Gaussian blobs plus a uniform background."""
    g = _rng(seed, 5)
    centres = g.random((n_centres, 3))
    n_bg = int(round(frac_background * n))
    n_blob = n - n_bg
    which = g.integers(0, n_centres, n_blob)
    pts = centres[which] + sigma * g.standard_normal((n_blob, 3))
    bad = np.any((pts < 0.0) | (pts >= 1.0), axis=1)
    while bad.any():
        k = int(bad.sum())
        w2 = g.integers(0, n_centres, k)
        pts[bad] = centres[w2] + sigma * g.standard_normal((k, 3))
        bad = np.any((pts < 0.0) | (pts >= 1.0), axis=1)
    bg = g.random((n_bg, 3))
    x = np.concatenate([pts, bg], axis=0)
    return x[g.permutation(n)]


def lognormal_sizes(n_systems: int, seed: int, mu: float = float(np.log(1e4)),
                    sigma: float = 1.0, lo: int = 1000, hi: int = 100000) -> np.ndarray:
    """System sizes for the batched workload (int64)."""
    s = _rng(seed, 6).lognormal(mu, sigma, n_systems)
    return np.clip(np.round(s), lo, hi).astype(np.int64)


def min_pair_distance_ok(x: np.ndarray, tol: float = 0.0) -> bool:
    """True when no two points coincide (used to reject degenerate draws)."""
    if len(x) < 2:
        return True
    u = np.unique(x, axis=0)
    return len(u) == len(x)


# ---------------------------------------------------------------------------
# The five evaluated workloads (sizes as stated for each configuration).
# ---------------------------------------------------------------------------

def stokeslet_uniform(n: int, seed: int):
    """Stokeslet workload: uniform points in [0,1)^3, forces N(0,1)^3."""
    return uniform_points(n, seed), normal_vectors(n, seed)


def stresslet_blobs(n: int, seed: int):
    """Stresslet workload: clustered points, f ~ N(0,1)^3, q random unit vectors."""
    return blob_points(n, seed), normal_vectors(n, seed), unit_vectors(n, seed)


def rotlet_uniform(n: int, seed: int):
    """Rotlet workload: uniform points, torques N(0,1)^3, upstream grads N(0,1)^3."""
    x = uniform_points(n, seed)
    t = normal_vectors(n, seed)
    g = _rng(seed, 7).standard_normal((n, 3))
    return x, t, g


def batched_systems(n_systems: int, n_rhs: int, seed: int):
    """List of (x, f) per system, f of shape (N_s, n_rhs, 3), each in [0,1)^3."""
    sizes = lognormal_sizes(n_systems, seed)
    out = []
    for s, n in enumerate(sizes):
        x = uniform_points(int(n), seed * 1000 + s + 1)
        f = _rng(seed * 1000 + s + 1, 8).standard_normal((int(n), n_rhs, 3))
        out.append((x, f))
    return out
