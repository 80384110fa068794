"""Seeded synthetic inputs shaped like the paper's workloads.

This module serves both the CUDA path and the CPU oracle and therefore holds
none of the method's arithmetic: it only draws initial positions (and replica
sizes) from numpy's own generator.  Every draw is float64; FP32 runs cast the
same bits down, so both sides start from identical values.

Workloads (the paper runs on synthetic particle systems only; no dataset):
  - ``dyson``: N(0,1) i.i.d. on the line (Dyson Brownian motion, Sec. 4.2).
  - ``semicircle``: density sqrt(R^2 - x^2) (Sec. 4.1 and eq. "analyticaldis"),
    drawn as the first coordinate of a uniform point of the disc of radius R.
  - ``sphere``: uniform points on S^2 (Thomson problem, Sec. 5.1).
  - ``unit_cube``: U[0,1]^d (opinion dynamics, Sec. 5.2).
  - ``gaussian``: N(0, I_d).
  - ``mixture``: equal-weight isotropic Gaussian mixture with means on a circle.
  - ``replica_sizes``: log-uniform integer sizes in [lo, hi].
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), 0x52424D31]))


def dyson(n: int, seed: int = 0) -> np.ndarray:
    return _rng(seed).standard_normal((n, 1))


def semicircle(n: int, radius: float = 2.0, seed: int = 0) -> np.ndarray:
    g = _rng(seed)
    r = radius * np.sqrt(g.random(n))
    theta = 2.0 * np.pi * g.random(n)
    return (r * np.cos(theta)).reshape(n, 1)


def sphere(n: int, d: int = 3, seed: int = 0) -> np.ndarray:
    x = _rng(seed).standard_normal((n, d))
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def unit_cube(n: int, d: int = 2, seed: int = 0) -> np.ndarray:
    return _rng(seed).random((n, d))


def gaussian(n: int, d: int = 3, seed: int = 0) -> np.ndarray:
    return _rng(seed).standard_normal((n, d))


def mixture(n: int, d: int = 2, components: int = 4, radius: float = 3.0, std: float = 0.5,
            seed: int = 0) -> np.ndarray:
    g = _rng(seed)
    c = g.integers(0, components, size=n)
    ang = 2.0 * np.pi * c / components
    means = np.zeros((n, d))
    means[:, 0] = radius * np.cos(ang)
    if d > 1:
        means[:, 1] = radius * np.sin(ang)
    return means + std * g.standard_normal((n, d))


def replica_sizes(r: int, lo: int = 256, hi: int = 65536, seed: int = 0) -> np.ndarray:
    u = _rng(seed).random(r)
    n = np.floor(lo * (hi / lo) ** u).astype(np.int64)
    return np.clip(n, lo, hi)
