"""Seeded synthetic inputs shaped like the paper's experiments.

This module holds no arithmetic of the method: it only draws point clouds and
right-hand sides, so that the CUDA path and the CPU oracle see identical inputs.
All generators use numpy's PCG64 (``numpy.random.default_rng(seed)``).

Workloads (Sec. 5.1 uses uniform random points in B = [-1, 1]^3 and a random x):

* ``grid(n)``          -- cell-centred n^3 grid, x_i = -1 + (i + 1/2) h, h = 2/n.
* ``uniform(N, seed)`` -- N points uniform in [-1, 1]^3.
* ``jittered_grid(n, seed)`` -- cell-centred grid plus U(-h/4, h/4) per axis.
* ``sphere(N, seed)``  -- N points uniform on the unit sphere (normalised Gaussians).
* ``rhs_uniform`` / ``rhs_normal`` -- N x nrhs right-hand sides, column-major.
"""
from __future__ import annotations

import numpy as np


def grid(n: int) -> np.ndarray:
    h = 2.0 / n
    c = -1.0 + (np.arange(n, dtype=np.float64) + 0.5) * h
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    return np.ascontiguousarray(np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1))


def uniform(N: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(-1.0, 1.0, size=(N, 3)))


def jittered_grid(n: int, seed: int) -> np.ndarray:
    h = 2.0 / n
    rng = np.random.default_rng(seed)
    p = grid(n)
    p += rng.uniform(-0.25 * h, 0.25 * h, size=p.shape)
    return np.ascontiguousarray(p)


def sphere(N: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(size=(N, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return np.ascontiguousarray(g)


def rhs_uniform(N: int, nrhs: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, size=(nrhs, N)).T)


def rhs_normal(N: int, nrhs: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal(size=(nrhs, N)).T)


def sample_rows(N: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    count = min(count, N)
    return np.sort(rng.choice(N, size=count, replace=False)).astype(np.int64)
