"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds none of the block-Vecchia arithmetic: it only draws locations,
standard-normal vectors and parameter perturbations.  Observations y (which need the
covariance model) are made by the method itself: by the library's block-Vecchia sampler
on the product side, or by the oracle's draws inside the tests.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) in counter
form, draw c of stream s = finaliser(s + (c + 1) * 0x9e3779b97f4a7c15), so every input
is a pure function of its seed.

Workload shapes follow the paper's studies (irregular locations in the unit square,
Sec. 3.1-3.2; million-point 3D profiles scaled to the unit cube, Sec. 4).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def stream(seed: int, tag: int) -> int:
    """Independent stream id for (seed, tag)."""
    return int(splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF), np.array([tag], np.uint64))[0])


def splitmix64(s, counters: np.ndarray) -> np.ndarray:
    """Vectorised SplitMix64 draws number `counters` of stream `s`."""
    with np.errstate(over="ignore"):
        z = np.uint64(s) + (counters.astype(np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, tag: int, count: int) -> np.ndarray:
    """count doubles in [0, 1) with 53 random bits each."""
    r = splitmix64(stream(seed, tag), np.arange(count, dtype=np.uint64))
    return (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, tag: int, count: int) -> np.ndarray:
    """count standard normals by the Box-Muller transform."""
    u = uniform01(seed, tag, 2 * count)
    u1, u2 = 1.0 - u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def locs_uniform(n: int, d: int, seed: int) -> np.ndarray:
    """n irregular locations uniform in [0, 1]^d (row-major n x d)."""
    return uniform01(seed, 1, n * d).reshape(n, d)


def locs_levels(n_sites: int, n_levels: int, seed: int, jitter: float = 0.2) -> np.ndarray:
    """3D profile: n_sites uniform (x, y) sites times n_levels heights; level k sits at
    (k + 1/2)/n_levels, jittered per point by U(-jitter, jitter)/n_levels."""
    xy = uniform01(seed, 2, n_sites * 2).reshape(n_sites, 2)
    j = uniform01(seed, 3, n_sites * n_levels) * 2.0 - 1.0
    z = (np.arange(n_levels)[None, :] + 0.5 + jitter * j.reshape(n_sites, n_levels)) / n_levels
    out = np.empty((n_sites * n_levels, 3))
    out[:, 0] = np.repeat(xy[:, 0], n_levels)
    out[:, 1] = np.repeat(xy[:, 1], n_levels)
    out[:, 2] = z.ravel()
    return out


def perturb_factors(seed: int, count: int, lo: float = 0.8, hi: float = 1.2) -> np.ndarray:
    """count x 3 multiplicative factors U(lo, hi) for (sigma^2, beta, tau^2)."""
    return lo + (hi - lo) * uniform01(seed, 4, 3 * count).reshape(count, 3)


def log_uniform(seed: int, tag: int, count: int, lo: float, hi: float) -> np.ndarray:
    u = uniform01(seed, tag, count)
    return np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))


def dataset_sizes(seed: int, count: int, lo: int = 5000, hi: int = 50000) -> np.ndarray:
    """Per-dataset sizes, log-uniform in [lo, hi]."""
    return np.floor(log_uniform(seed, 5, count, lo, hi)).astype(np.int64)


def theta_draws(seed: int, count: int):
    """Per-dataset parameters drawn as in the warm-start training design:
    sigma^2 in [0.5, 2], beta in [0.02, 0.3], tau^2 in [1e-4, 1e-1] (log-uniform) and
    nu uniform over {0.5, 1.5, 2.5}.  Returns an array (count, 4): sigma2, beta, nugget, nu."""
    s2 = log_uniform(seed, 6, count, 0.5, 2.0)
    be = log_uniform(seed, 7, count, 0.02, 0.3)
    tn = log_uniform(seed, 8, count, 1e-4, 1e-1)
    nu = np.array([0.5, 1.5, 2.5])[np.minimum((uniform01(seed, 9, count) * 3).astype(int), 2)]
    return np.stack([s2, be, tn, nu], axis=1)
