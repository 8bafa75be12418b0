"""Seeded synthetic rigid-body workloads (bead shells, ellipsoids, batches).

This module only draws random inputs; it holds none of the method's
arithmetic and imports neither the CUDA binding nor the oracle, so both sides
can share it.  All generators use ``numpy.random.default_rng(seed)`` (PCG64).

Shapes follow the workloads named for this library:

* ``shell_body``      -- one body: directions uniform on the sphere times a
  radius, plus isotropic Gaussian jitter per coordinate (single-body case,
  n = 256, radius 2.0, sigma 0.05).
* ``ellipsoid_body``  -- one large body: points (a u_x, b u_y, c u_z) + eps u
  with u uniform on the sphere and eps ~ N(0, sigma^2) radial jitter
  (n = 2^20, semi-axes (3, 2, 1) sqrt(n)/100, sigma 0.01).
* ``shell_batch``     -- many bodies with log-uniform bead counts, each a
  jittered shell of radius 0.1 sqrt(n_j) (jitter 0.025 x radius) centred at
  a uniform point of a 100^3 box (m = 2000, n_j in [50, 5000]).
* ``uniform_batch``   -- many bodies with uniformly distributed counts
  (multi-right-hand-side case: m = 500, n_j in [500, 2000]).
* ``random_rigid_motions`` -- per-step uniform random rotations (normalised
  Gaussian quaternions) and Gaussian translations for a Brownian-dynamics
  style loop.

Coordinates are float64 structure-of-arrays (x, y, z); body offsets are an
int64 CSR array of length m + 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Batch:
    off: np.ndarray  # int64 [m + 1]
    x: np.ndarray    # float64 [N]
    y: np.ndarray
    z: np.ndarray

    @property
    def m(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def N(self) -> int:
        return int(self.off[-1])

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.off)

    @property
    def n_residues(self) -> int:
        return 3 * self.N - 6 * self.m

    def body(self, j: int):
        a, b = int(self.off[j]), int(self.off[j + 1])
        return self.x[a:b], self.y[a:b], self.z[a:b]


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return u


def shell_body(n: int = 256, radius: float = 2.0, sigma: float = 0.05, seed: int = 0,
               centre=(0.0, 0.0, 0.0)) -> Batch:
    rng = np.random.default_rng(seed)
    p = _unit_vectors(rng, n) * radius + rng.standard_normal((n, 3)) * sigma
    p += np.asarray(centre, dtype=np.float64)
    return Batch(np.array([0, n], np.int64), p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy())


def ellipsoid_body(n: int = 1 << 20, sigma: float = 0.01, seed: int = 0) -> Batch:
    rng = np.random.default_rng(seed)
    s = np.sqrt(n) / 100.0
    axes = np.array([3.0, 2.0, 1.0]) * s
    u = _unit_vectors(rng, n)
    eps = rng.standard_normal(n) * sigma
    p = u * axes + eps[:, None] * u
    return Batch(np.array([0, n], np.int64), p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy())


def _shells(rng: np.random.Generator, sizes: np.ndarray, box: float, jitter_ratio: float):
    m = sizes.shape[0]
    off = np.zeros(m + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    N = int(off[-1])
    pts = np.empty((N, 3))
    centres = rng.uniform(0.0, box, size=(m, 3))
    for j in range(m):
        n = int(sizes[j])
        r = 0.1 * np.sqrt(n)
        p = _unit_vectors(rng, n) * r + rng.standard_normal((n, 3)) * (jitter_ratio * r)
        pts[off[j]:off[j + 1]] = p + centres[j]
    return Batch(off, pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy())


def shell_batch(m: int = 2000, nmin: int = 50, nmax: int = 5000, seed: int = 0,
                box: float = 100.0, jitter_ratio: float = 0.025) -> Batch:
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=m))).astype(np.int64)
    sizes = np.clip(sizes, max(nmin, 3), nmax)
    return _shells(rng, sizes, box, jitter_ratio)


def uniform_batch(m: int = 500, nmin: int = 500, nmax: int = 2000, seed: int = 0,
                  box: float = 100.0, jitter_ratio: float = 0.025) -> Batch:
    rng = np.random.default_rng(seed)
    sizes = rng.integers(nmin, nmax + 1, size=m).astype(np.int64)
    return _shells(rng, sizes, box, jitter_ratio)


def fixed_batch(m: int = 1000, n: int = 1000, seed: int = 0, box: float = 100.0,
                jitter_ratio: float = 0.025) -> Batch:
    rng = np.random.default_rng(seed)
    return _shells(rng, np.full(m, n, np.int64), box, jitter_ratio)


def vectors(rng_seed: int, length: int, k: int = 1) -> np.ndarray:
    """k i.i.d. N(0, 1) vectors of the given length, shape (k, length)."""
    rng = np.random.default_rng(rng_seed)
    return rng.standard_normal((k, length))


def random_rigid_motions(m: int, steps: int, seed: int = 0, sigma_t: float = 0.1):
    """Unit quaternions (steps, m, 4) from normalised N(0, I_4) draws and
    translations (steps, m, 3) ~ N(0, sigma_t^2)."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((steps, m, 4))
    q /= np.linalg.norm(q, axis=2, keepdims=True)
    t = rng.standard_normal((steps, m, 3)) * sigma_t
    return q, t


def interleave(x: np.ndarray, y: np.ndarray, z: np.ndarray) -> np.ndarray:
    """SoA planes -> the paper's bead ordering [v_1; v_2; ...] (3i + a)."""
    return np.stack([x, y, z], axis=1).reshape(-1)


def planes(v: np.ndarray) -> np.ndarray:
    """The paper's bead ordering -> SoA planes, shape (3, N)."""
    return np.ascontiguousarray(v.reshape(-1, 3).T)
