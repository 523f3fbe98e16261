"""Proxy surfaces, interpolative decompositions and Algorithm 1 — oracle.

Test infrastructure only.

Section 2.1: for a box B with index set I_B, a column ID of the stacked
matrix [A_{F,B}; A_{B,F}^*] splits I_B into skeleton S and redundant R
indices with A_{.,R} ~= A_{.,S} T. The far field F is replaced by a proxy
surface: Chebyshev points on the boundary of a box of side 2.95 a centred on
B (a = side of B). For a kernel with G(x, y) = G(y, x) the stacked matrix is
[G(P, I_B); conj(G(P, I_B))]; for real kernels the second half repeats the
first and is dropped.

Readings where the paper is silent:
* proxy points: p first-kind Chebyshev nodes cos((2k-1) pi / (2p)) per edge
  of the square (4p points) or a p x p tensor grid per face of the cube
  (6 p^2 points), scaled to the proxy box (no point lies on an edge);
* rank rule: the ID keeps the leading k pivots with |R_jj| > tol |R_00|
  of a column-pivoted QR (the paper's greedy CPQR, Section 2.1);
* T = R_11^{-1} R_12, the standard ID coefficients.

Algorithm 1 runs the ID level by level from the leaves up; a tree box's
index set is the concatenation of its children's skeletons (child order).
The level-1 ID is not computed: Algorithm 2 never uses level-1 outgoing
skeleton charges (there is no level-0 translation), so level-1 boxes keep
S = I_B and an empty T.

Layout of one box's ID (shared with the plan format): ``idx`` = the global
point indices of I_B in "slot order" (leaf: ascending point index; tree box:
children's skeletons concatenated); ``piv`` = a permutation of
0..|I_B|-1 whose first k entries are the positions of S (in pivot order) and
the rest the positions of R; ``T`` = k x |R|.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import kernels
from .tree import Tree

PROXY_SCALE = 2.95
DEFAULT_P = {2: 32, 3: 12}


def chebyshev_nodes(p: int) -> np.ndarray:
    k = np.arange(1, p + 1)
    return np.cos((2 * k - 1) * np.pi / (2 * p))


def proxy_points(center: np.ndarray, a: float, dim: int, p: int) -> np.ndarray:
    """Points on the boundary of the box of side 2.95 a centred at `center`."""
    h = 0.5 * PROXY_SCALE * a
    t = h * chebyshev_nodes(p)
    pts = []
    if dim == 2:
        for axis in range(2):
            for sgn in (-1.0, 1.0):
                blk = np.zeros((p, 2))
                blk[:, axis] = sgn * h
                blk[:, 1 - axis] = t
                pts.append(blk)
    else:
        g1, g2 = np.meshgrid(t, t, indexing="ij")
        g1 = g1.ravel()
        g2 = g2.ravel()
        for axis in range(3):
            others = [d for d in range(3) if d != axis]
            for sgn in (-1.0, 1.0):
                blk = np.zeros((p * p, 3))
                blk[:, axis] = sgn * h
                blk[:, others[0]] = g1
                blk[:, others[1]] = g2
                pts.append(blk)
    return center[None, :] + np.concatenate(pts, axis=0)


def proxy_matrix(kind: str, proxy: np.ndarray, xb: np.ndarray, kappa: float) -> np.ndarray:
    g = kernels.kernel_matrix(kind, proxy, xb, kappa)
    if np.iscomplexobj(g):
        return np.vstack([g, np.conj(g)])
    return g


def interpolative_decomposition(m: np.ndarray, tol: float, keep_all: bool = False):
    """Column ID by column-pivoted QR: returns (piv, k, T) with
    M[:, piv[k:]] ~= M[:, piv[:k]] @ T."""
    n = m.shape[1]
    if keep_all:
        return np.arange(n), n, np.zeros((n, 0), dtype=m.dtype)
    _, r, piv = scipy.linalg.qr(m, mode="economic", pivoting=True)
    d = np.abs(np.diag(r))
    if d.shape[0] == 0 or d[0] == 0.0:
        return piv, n, np.zeros((n, 0), dtype=m.dtype)
    k = int(np.count_nonzero(d > tol * d[0]))
    k = max(k, 1)
    if k >= n:
        return piv, n, np.zeros((n, 0), dtype=m.dtype)
    t = scipy.linalg.solve_triangular(r[:k, :k], r[:k, k:n])
    return piv, k, t


class Skeletons:
    """Per-box index sets and IDs produced by Algorithm 1 on a Tree."""

    def __init__(self, tree: Tree, kind: str, tol: float, kappa: float = 0.0,
                 proxy_p: int | None = None, keep_all: bool = False):
        self.tree = tree
        self.kind = kind
        self.kappa = float(kappa)
        self.tol = float(tol)
        self.proxy_p = int(proxy_p or DEFAULT_P[tree.dim])
        nb = tree.n_boxes
        self.idx = [None] * nb
        self.piv = [None] * nb
        self.k = np.zeros(nb, dtype=np.int64)
        self.T = [None] * nb
        cdtype = np.complex128 if kernels.is_complex(kind) else np.float64
        for lvl in range(tree.n_levels, 0, -1):
            for b in tree.boxes_at[lvl]:
                if tree.is_leaf[b]:
                    idx = tree.points[b]
                else:
                    idx = np.concatenate([self.skel(c) for c in tree.children[b]])
                self.idx[b] = idx
                if lvl == 1:
                    self.piv[b], self.k[b] = np.arange(idx.shape[0]), idx.shape[0]
                    self.T[b] = np.zeros((idx.shape[0], 0), dtype=cdtype)
                    continue
                prox = proxy_points(tree.box_center(b), tree.box_side(b), tree.dim, self.proxy_p)
                m = proxy_matrix(kind, prox, tree.x[idx], self.kappa)
                piv, k, t = interpolative_decomposition(m, self.tol, keep_all)
                self.piv[b], self.k[b], self.T[b] = piv, k, t.astype(cdtype)
        if tree.n_levels == 0:
            self.idx[0] = tree.points[0]
            self.piv[0] = np.arange(tree.n)
            self.k[0] = tree.n
            self.T[0] = np.zeros((tree.n, 0), dtype=cdtype)

    def skel(self, b: int) -> np.ndarray:
        """Global point indices of S_b, in pivot order."""
        return self.idx[b][self.piv[b][: self.k[b]]]

    def k_max(self) -> int:
        lv = self.tree.level
        ks = [int(self.k[b]) for b in range(self.tree.n_boxes) if lv[b] >= 2]
        return max(ks) if ks else 0
