"""Kernel functions G(x, y) — oracle (test infrastructure only).

Laplace (Eq. (2)):   2D  G = -log|x-y| / (2 pi),   3D  G = 1 / (4 pi |x-y|).
Helmholtz 3D (Eq. (5)): the paper prints (1/4) e^{i kappa r} / r; this
library uses the free-space normalisation e^{i kappa r} / (4 pi r) (a global
scale; the method is unchanged).
Helmholtz 2D (Section 5, the 2D Helmholtz experiments): the free-space
fundamental solution G = (i/4) H_0^(1)(kappa r), with the Hankel function
taken from scipy.special (a library routine).

The matrix A has zero diagonal (Section 1, below Eq. (3)); coincident points
(r == 0) are given G = 0 as well, the same rule as the diagonal.

``poly2`` is not from the paper: G(x, y) = (1 + x.y)^2 is exactly low rank
(rank 6 in 2D, 10 in 3D) away from the diagonal, so an interpolative
decomposition of it is exact and the skeleton apply must reproduce the direct
sum to rounding. It is used only to pin the oracle's plumbing.
"""
from __future__ import annotations

import numpy as np

KINDS = ("laplace2d", "laplace3d", "helmholtz3d", "helmholtz2d", "poly2")


def is_complex(kind: str) -> bool:
    return kind in ("helmholtz3d", "helmholtz2d")


def kernel_dim(kind: str) -> int | None:
    return {"laplace2d": 2, "laplace3d": 3, "helmholtz3d": 3, "helmholtz2d": 2}.get(kind)


def _hankel_2d(kr: np.ndarray) -> np.ndarray:
    from scipy.special import hankel1
    return 0.25j * hankel1(0, kr)


def kernel_matrix(kind: str, xt: np.ndarray, xs: np.ndarray, kappa: float = 0.0) -> np.ndarray:
    """Dense block G(xt_i, xs_j) for targets xt (m x d) and sources xs (n x d)."""
    xt = np.asarray(xt, dtype=np.float64)
    xs = np.asarray(xs, dtype=np.float64)
    if kind == "poly2":
        g = (1.0 + xt @ xs.T) ** 2
        diff = xt[:, None, :] - xs[None, :, :]
        r2 = np.einsum("ijk,ijk->ij", diff, diff)
        g[r2 == 0.0] = 0.0
        return g
    diff = xt[:, None, :] - xs[None, :, :]
    r = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    if kind == "laplace2d":
        g = -np.log(rs) / (2.0 * np.pi)
    elif kind == "laplace3d":
        g = 1.0 / (4.0 * np.pi * rs)
    elif kind == "helmholtz3d":
        g = np.exp(1j * kappa * rs) / (4.0 * np.pi * rs)
    elif kind == "helmholtz2d":
        g = _hankel_2d(kappa * rs)
    else:
        raise ValueError(kind)
    g[zero] = 0.0
    return g


def kernel_scalar(kind: str, r: float, kappa: float = 0.0):
    """G as a function of the distance r (r > 0) for the radial kernels."""
    if kind == "laplace2d":
        return -np.log(r) / (2.0 * np.pi)
    if kind == "laplace3d":
        return 1.0 / (4.0 * np.pi * r)
    if kind == "helmholtz3d":
        return np.exp(1j * kappa * r) / (4.0 * np.pi * r)
    if kind == "helmholtz2d":
        return complex(_hankel_2d(np.array(kappa * r)))
    raise ValueError(kind)
