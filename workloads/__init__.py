"""Seeded synthetic point clouds for the FAMST hot path.

This module only draws inputs. It holds none of the method's arithmetic, so
both the CUDA path and the CPU oracle may be fed from it.

Every generator returns a C-contiguous float32 array of shape (n, d) and is a
pure function of its seed (numpy ``default_rng``). Rows are shuffled, as
scikit-learn's ``make_blobs`` does, so cluster members are not contiguous in
id order.

Workloads (the paper's experiments use ``make_blobs`` style mixtures and real
datasets that are not available here; these stand in for them):

* ``blobs_small``   n=2,000, d=16, 10 isotropic clusters, sigma=1, k=10, lambda=5
* ``blobs_100k``    n=100,000, d=128, 50 clusters, sigma_c ~ U[0.5, 2], k=16, lambda=5
* ``sphere_1m``     n=1,000,000, d=128, 1,000 clusters of unit vectors, k=32, lambda=10
* ``moons_50k``     n=50,000, d=64, two moons embedded in 64-D, noise sd 0.05, k=16, lambda=5
* ``batch_256``     256 clouds, n_b ~ U{500..20000}, d_b in {3, 32, 128}, 5-20 clusters, k=16, lambda=5
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "Workload", "WORKLOADS", "get", "blobs", "unit_sphere_mixture",
    "two_moons", "batch_clouds", "integer_grid", "collinear", "regular_polygon",
    "with_duplicates",
]


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    k: int
    lam: int
    seed: int
    kind: str

    def points(self, n: int | None = None) -> np.ndarray:
        """Draw the cloud; ``n`` overrides the size with the same recipe."""
        n = self.n if n is None else n
        if self.kind == "blobs_small":
            return blobs(n, self.d, centres=10, sigma=(1.0, 1.0), seed=self.seed)
        if self.kind == "blobs_100k":
            return blobs(n, self.d, centres=50, sigma=(0.5, 2.0), seed=self.seed)
        if self.kind == "sphere_1m":
            return unit_sphere_mixture(n, self.d, centres=1000, sigma=0.02,
                                       seed=self.seed)
        if self.kind == "moons_50k":
            return two_moons(n, self.d, noise=0.05, seed=self.seed)
        raise ValueError(self.kind)


WORKLOADS = {
    "blobs_small": Workload("blobs_small", 2000, 16, 10, 5, 0, "blobs_small"),
    "blobs_100k": Workload("blobs_100k", 100_000, 128, 16, 5, 1, "blobs_100k"),
    "sphere_1m": Workload("sphere_1m", 1_000_000, 128, 32, 10, 2, "sphere_1m"),
    "moons_50k": Workload("moons_50k", 50_000, 64, 16, 5, 3, "moons_50k"),
}


def get(name: str) -> Workload:
    return WORKLOADS[name]


def _even_split(n: int, c: int) -> np.ndarray:
    sizes = np.full(c, n // c, dtype=np.int64)
    sizes[: n % c] += 1
    return sizes


def blobs(n: int, d: int, centres: int, sigma: tuple[float, float],
          seed: int, box: float = 10.0) -> np.ndarray:
    """Isotropic Gaussian mixture: centres ~ U[-box, box]^d, per-cluster
    standard deviation ~ U[sigma[0], sigma[1]], clusters split evenly."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-box, box, size=(centres, d))
    s = rng.uniform(sigma[0], sigma[1], size=centres)
    sizes = _even_split(n, centres)
    lab = np.repeat(np.arange(centres), sizes)
    x = c[lab] + rng.standard_normal((n, d)) * s[lab, None]
    x = x[rng.permutation(n)]
    return np.ascontiguousarray(x, dtype=np.float32)


def unit_sphere_mixture(n: int, d: int, centres: int, sigma: float,
                        seed: int) -> np.ndarray:
    """Unit vectors: centre c ~ N(0, I) normalised, point =
    normalise(c + N(0, sigma^2 I)); clusters split evenly."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((centres, d))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    sizes = _even_split(n, centres)
    lab = np.repeat(np.arange(centres), sizes)
    out = np.empty((n, d), dtype=np.float32)
    step = 1 << 17
    for a in range(0, n, step):
        b = min(n, a + step)
        x = c[lab[a:b]] + sigma * rng.standard_normal((b - a, d))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[a:b] = x
    return np.ascontiguousarray(out[rng.permutation(n)])


def two_moons(n: int, d: int, noise: float, seed: int) -> np.ndarray:
    """Two interleaved half circles in 2-D, embedded in d dimensions by a
    seeded random orthonormal d x 2 matrix, plus N(0, noise^2) in every
    dimension."""
    rng = np.random.default_rng(seed)
    na = n // 2
    nb = n - na
    ta = rng.uniform(0.0, np.pi, na)
    tb = rng.uniform(0.0, np.pi, nb)
    a = np.stack([np.cos(ta), np.sin(ta)], axis=1)
    b = np.stack([1.0 - np.cos(tb), 0.5 - np.sin(tb)], axis=1)
    p2 = np.concatenate([a, b], axis=0)
    q, _ = np.linalg.qr(rng.standard_normal((d, 2)))
    x = p2 @ q.T + noise * rng.standard_normal((n, d))
    x = x[rng.permutation(n)]
    return np.ascontiguousarray(x, dtype=np.float32)


def batch_clouds(count: int = 256, base_seed: int = 1000,
                 n_range: tuple[int, int] = (500, 20000),
                 dims: tuple[int, ...] = (3, 32, 128),
                 centre_range: tuple[int, int] = (5, 20)) -> list[np.ndarray]:
    """Many Gaussian-mixture clouds of uneven size; cloud b uses seed
    base_seed + b for n_b, d_b, its centre count and its points."""
    out = []
    for b in range(count):
        rng = np.random.default_rng(base_seed + b)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        d = int(dims[int(rng.integers(0, len(dims)))])
        c = int(rng.integers(centre_range[0], centre_range[1] + 1))
        out.append(blobs(n, d, centres=c, sigma=(1.0, 1.0),
                         seed=int(rng.integers(0, 2**31 - 1))))
    return out


# ---- small structured clouds used by the tests -------------------------

def integer_grid(m: int, d: int = 2) -> np.ndarray:
    """The m x m unit grid (d=2) padded with zero coordinates up to d."""
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), indexing="ij"), -1)
    g = g.reshape(-1, 2).astype(np.float32)
    out = np.zeros((g.shape[0], d), dtype=np.float32)
    out[:, :2] = g
    return out


def collinear(n: int, d: int, seed: int) -> np.ndarray:
    """n distinct integer positions on a line through the origin along the
    first axis (other coordinates zero), in shuffled order."""
    rng = np.random.default_rng(seed)
    pos = rng.choice(np.arange(-4 * n, 4 * n), size=n, replace=False)
    out = np.zeros((n, d), dtype=np.float32)
    out[:, 0] = pos
    return out


def regular_polygon(n: int, radius: float = 10.0) -> np.ndarray:
    """Vertices of a regular n-gon in the plane."""
    a = 2.0 * np.pi * np.arange(n) / n
    return np.ascontiguousarray(
        np.stack([radius * np.cos(a), radius * np.sin(a)], 1), dtype=np.float32)


def with_duplicates(x: np.ndarray, copies: int, seed: int) -> np.ndarray:
    """Append exact copies of randomly chosen rows (zero-distance pairs)."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, x.shape[0], size=copies)
    y = np.concatenate([x, x[idx]], axis=0)
    return np.ascontiguousarray(y[rng.permutation(y.shape[0])], dtype=np.float32)
